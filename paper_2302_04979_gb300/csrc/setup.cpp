// Host-side FP64 setup: univariate bases, Gauss rules, pairing matrices and
// their banded LU, element masses.  See setup.h for the conventions.
#include "setup.h"

#include "smx.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace smx {

// Component kinds (x, y, z) per field, Sec. 2.3 / Sec. 4.1:
//   E (X^1_{h,0}): E_c has P1 along axis c, P0 along the others;
//   B (X^2_{h,0}): B_c has P0 along axis c, P1 along the others;
//   H (X~^1):      H_c has D1 along axis c, D0 along the others;
//   D (X~^2):      D_c has D0 along axis c, D1 along the others.
const int kFieldKinds[4][3][3] = {
    {{P1, P0, P0}, {P0, P1, P0}, {P0, P0, P1}},
    {{P0, P1, P1}, {P1, P0, P1}, {P1, P1, P0}},
    {{D1, D0, D0}, {D0, D1, D0}, {D0, D0, D1}},
    {{D0, D1, D1}, {D1, D0, D1}, {D1, D1, D0}},
};

int kind_degree(int kind, int p) {
    switch (kind) {
        case P0: return p;
        case P1: return p - 1;
        case D0: return p - 1;
        default: return p - 2;
    }
}

int kind_dim(int kind, int p, int nel) {
    const int n = nel + p;
    return (kind == P0 || kind == D1) ? n - 2 : n - 1;
}

int kind_offset(int kind) { return kind == P0 ? -1 : 0; }

static bool kind_is_cs(int kind) { return kind == P1 || kind == D1; }

// Knot i of the open uniform knot vector of degree d: d+1 zeros, k/nel, d+1 ones.
static double knot(int d, int nel, int i) {
    const int k = i - d;
    if (k <= 0) return 0.0;
    if (k >= nel) return 1.0;
    return static_cast<double>(k) / nel;
}

void gauss_legendre01(int q, std::vector<double>& x, std::vector<double>& w) {
    x.assign(q, 0.0);
    w.assign(q, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < q; ++i) {
        double z = std::cos(pi * (i + 0.75) / (q + 0.5));  // guess for the (i+1)-th largest root
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            // P_q(z) and P_{q-1}(z) by the three-term recurrence
            double p0 = 1.0, p1 = z;
            if (q == 1) p1 = z;
            for (int k = 2; k <= q; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pq = (q == 1) ? z : p1;
            const double pqm1 = (q == 1) ? 1.0 : p0;
            dp = q * (z * pq - pqm1) / (z * z - 1.0);
            const double dz = pq / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute the derivative at the converged root
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= q; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        const double pq = (q == 1) ? z : p1, pqm1 = (q == 1) ? 1.0 : p0;
        dp = q * (z * pq - pqm1) / (z * z - 1.0);
        // map [-1,1] -> [0,1]; roots come out descending in z, so ascending in (1-z)/2 order is reversed
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // (2/((1-z^2) P'^2)) * 1/2
    }
}

void local_basis(int kind, int p, int nel, int e, double x, double* out) {
    const int d = kind_degree(kind, p);
    const int s = d + e;  // knot span: knot(s) <= x < knot(s+1)
    double left[16], right[16];
    out[0] = 1.0;
    for (int j = 1; j <= d; ++j) {
        left[j] = x - knot(d, nel, s + 1 - j);
        right[j] = knot(d, nel, s + j) - x;
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            const double tmp = out[r] / (right[r + 1] + left[j - r]);
            out[r] = saved + right[r + 1] * tmp;
            saved = left[j - r] * tmp;
        }
        out[j] = saved;
    }
    if (kind_is_cs(kind)) {
        for (int r = 0; r <= d; ++r) {
            const int i = e + r;  // full index
            out[r] *= (d + 1) / (knot(d, nel, i + d + 1) - knot(d, nel, i));
        }
    }
}

std::vector<double> pairing_matrix(int row_kind, int col_kind, int p, int nel) {
    const int nr = kind_dim(row_kind, p, nel), nc = kind_dim(col_kind, p, nel);
    const int dr = kind_degree(row_kind, p), dc = kind_degree(col_kind, p);
    const int q = p + 1;
    std::vector<double> gx, gw;
    gauss_legendre01(q, gx, gw);
    std::vector<double> A(static_cast<size_t>(nr) * nc, 0.0);
    double vr[16], vc[16];
    for (int e = 0; e < nel; ++e) {
        for (int k = 0; k < q; ++k) {
            const double x = (e + gx[k]) / nel, w = gw[k] / nel;
            local_basis(row_kind, p, nel, e, x, vr);
            local_basis(col_kind, p, nel, e, x, vc);
            for (int a = 0; a <= dr; ++a) {
                const int i = e + a + kind_offset(row_kind);
                if (i < 0 || i >= nr) continue;
                for (int b = 0; b <= dc; ++b) {
                    const int j = e + b + kind_offset(col_kind);
                    if (j < 0 || j >= nc) continue;
                    A[static_cast<size_t>(i) * nc + j] += w * vr[a] * vc[b];
                }
            }
        }
    }
    return A;
}

bool band_lu(const std::vector<double>& A0, int n, int kl, int ku, BandLU& out) {
    std::vector<double> A(A0);
    double amax = 0.0;
    for (double v : A) amax = std::max(amax, std::fabs(v));
    // Doolittle elimination without pivoting, restricted to the band
    for (int k = 0; k < n; ++k) {
        const double piv = A[static_cast<size_t>(k) * n + k];
        if (!(std::fabs(piv) > 1e-12 * amax)) return false;
        for (int i = k + 1; i <= std::min(n - 1, k + kl); ++i) {
            const double l = A[static_cast<size_t>(i) * n + k] / piv;
            A[static_cast<size_t>(i) * n + k] = l;
            for (int j = k + 1; j <= std::min(n - 1, k + ku); ++j)
                A[static_cast<size_t>(i) * n + j] -= l * A[static_cast<size_t>(k) * n + j];
        }
    }
    out.n = n;
    out.kl = kl;
    out.ku = ku;
    out.L.assign(static_cast<size_t>(n) * std::max(kl, 1), 0.0);
    out.U.assign(static_cast<size_t>(n) * std::max(ku, 1), 0.0);
    out.dinv.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        const double dii = A[static_cast<size_t>(i) * n + i];
        out.dinv[i] = 1.0 / dii;
        for (int k = 1; k <= kl; ++k)
            if (i - k >= 0) out.L[static_cast<size_t>(i) * kl + k - 1] = A[static_cast<size_t>(i) * n + i - k];
        for (int k = 1; k <= ku; ++k)
            if (i + k < n) out.U[static_cast<size_t>(i) * ku + k - 1] = A[static_cast<size_t>(i) * n + i + k] / dii;
    }
    return true;
}

std::vector<double> band_lu_dense(const BandLU& f) {
    const int n = f.n;
    std::vector<double> L(static_cast<size_t>(n) * n, 0.0), U(static_cast<size_t>(n) * n, 0.0);
    for (int i = 0; i < n; ++i) {
        L[static_cast<size_t>(i) * n + i] = 1.0;
        for (int k = 1; k <= f.kl; ++k)
            if (i - k >= 0) L[static_cast<size_t>(i) * n + i - k] = f.L[static_cast<size_t>(i) * f.kl + k - 1];
        const double dii = 1.0 / f.dinv[i];
        U[static_cast<size_t>(i) * n + i] = dii;
        for (int k = 1; k <= f.ku; ++k)
            if (i + k < n) U[static_cast<size_t>(i) * n + i + k] = f.U[static_cast<size_t>(i) * f.ku + k - 1] * dii;
    }
    std::vector<double> A(static_cast<size_t>(n) * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const double l = L[static_cast<size_t>(i) * n + k];
            if (l == 0.0) continue;
            for (int j = 0; j < n; ++j) A[static_cast<size_t>(i) * n + j] += l * U[static_cast<size_t>(k) * n + j];
        }
    return A;
}

std::vector<double> element_mass(int kind, int p, int nel, int e) {
    const int d = kind_degree(kind, p), m = d + 1, q = p + 1;
    std::vector<double> gx, gw;
    gauss_legendre01(q, gx, gw);
    std::vector<double> Me(static_cast<size_t>(m) * m, 0.0);
    double v[16];
    for (int k = 0; k < q; ++k) {
        const double x = (e + gx[k]) / nel, w = gw[k] / nel;
        local_basis(kind, p, nel, e, x, v);
        for (int a = 0; a < m; ++a)
            for (int b = 0; b < m; ++b) Me[a * m + b] += w * v[a] * v[b];
    }
    return Me;
}

// Map F and its Jacobian J (row-major, J[3 i + j] = dF_i / dxhat_j) at a parametric point.
void geometry_eval(int geom, double a, const double xh[3], double X[3], double J[9]) {
    for (int i = 0; i < 9; ++i) J[i] = (i % 4 == 0) ? 1.0 : 0.0;
    for (int i = 0; i < 3; ++i) X[i] = xh[i];
    if (geom == SMX_GEOM_SINE_BUMP) {
        const double pi = 3.14159265358979323846;
        const double sx = std::sin(pi * xh[0]), sy = std::sin(pi * xh[1]), sz = std::sin(pi * xh[2]);
        const double cx = std::cos(pi * xh[0]), cy = std::cos(pi * xh[1]), cz = std::cos(pi * xh[2]);
        const double S = sx * sy * sz;
        const double g[3] = {pi * cx * sy * sz, pi * sx * cy * sz, pi * sx * sy * cz};
        for (int i = 0; i < 3; ++i) {
            X[i] += a * S;
            for (int j = 0; j < 3; ++j) J[3 * i + j] += a * g[j];
        }
    }
}

double det3(const double J[9]) {
    return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
}

int geometry_eval_points(const GeomMap& g, int64_t n, const double* xh, double* X, double* J) {
    if (g.kind == SMX_GEOM_CALLBACK) {
        for (int64_t i = 0; i < 3 * n; ++i) X[i] = std::nan("");
        for (int64_t i = 0; i < 9 * n; ++i) J[i] = std::nan("");
        g.fn(n, xh, X, J, g.user);
    } else {
        for (int64_t i = 0; i < n; ++i) geometry_eval(g.kind, g.amp, xh + 3 * i, X + 3 * i, J + 9 * i);
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(X[3 * i + k])) return SMX_EGEOM;
        const double dj = det3(J + 9 * i);
        if (!std::isfinite(dj) || !(dj > 0.0)) return SMX_EGEOM;
    }
    return SMX_OK;
}

// Round an FP32 value to BF16, nearest even (IEEE rounding on the 16 dropped bits).
static uint16_t bf16_nearest(float f) {
    uint32_t u;
    std::memcpy(&u, &f, sizeof u);
    if ((u & 0x7F800000u) == 0x7F800000u) return static_cast<uint16_t>(u >> 16);  // inf / nan: not expected
    u += 0x7FFFu + ((u >> 16) & 1u);
    return static_cast<uint16_t>(u >> 16);
}

void digits_fixed(double v, int F, int nd, int* d) {
    uint64_t bits;
    std::memcpy(&bits, &v, sizeof bits);
    const int e = static_cast<int>((bits >> 52) & 0x7FF);
    const uint64_t frac = bits & 0xFFFFFFFFFFFFFull;
    const int eff = e ? e : 1;
    const uint64_t M = e ? (frac | (1ull << 52)) : frac;
    const int sh = F - eff - (8 * nd - 1 - 53);  // right shift of the significand (negative: left)
    uint64_t mag;
    if (sh <= 0) {
        mag = M << (-sh);
    } else {
        mag = sh >= 60 ? 0 : (M + (1ull << (sh - 1))) >> sh;
    }
    int64_t a = (bits >> 63) ? -static_cast<int64_t>(mag) : static_cast<int64_t>(mag);
    for (int t = nd - 1; t >= 1; --t) {
        const int dg = static_cast<int>((static_cast<uint64_t>(a) + 128) & 255) - 128;
        d[t] = dg;
        a = (a - dg) / 256;  // exact
    }
    d[0] = static_cast<int>(a);
}

void digit_split_operator(const std::vector<double>& B, int n, int npad, int nd, std::vector<uint16_t>& planes,
                          std::vector<int32_t>& rowexp) {
    const int r8 = (n + 7) / 8 * 8;
    const size_t col = static_cast<size_t>(r8) * 16, plane = static_cast<size_t>(npad / 16) * col;
    planes.assign(nd * plane, 0);
    rowexp.assign(r8, 1);
    std::vector<int> d(nd);
    for (int i = 0; i < n; ++i) {
        int F = 1;
        for (int k = 0; k < n; ++k) {
            uint64_t bits;
            std::memcpy(&bits, &B[static_cast<size_t>(i) * n + k], sizeof bits);
            F = std::max(F, static_cast<int>((bits >> 52) & 0x7FF));
        }
        rowexp[i] = F;
        for (int k = 0; k < n; ++k) {
            digits_fixed(B[static_cast<size_t>(i) * n + k], F, nd, d.data());
            for (int s = 0; s < nd; ++s)
                planes[s * plane + static_cast<size_t>(k / 16) * col + static_cast<size_t>(16) * i +
                       8 * (((k / 8) & 1) ^ ((i >> 2) & 1)) + k % 8] = bf16_nearest(static_cast<float>(d[s]));
        }
    }
}

}  // namespace smx
