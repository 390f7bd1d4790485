// L2 projection of a physical 2-form onto X~^2 or X^2_{h,0} (initial data and
// the source profile by projection, Sec. 5.1.1), on the host in FP64.
//
// A 2-form with physical vector proxy V is pulled back through the Piola map
// v = J vhat / det J (Sec. 2.2), so the right-hand side of the projection is
//   r_i = int_Omega V . (J vhat_i / det J) dx = int_Omegahat (J^T V) . vhat_i dxhat,
// and the coefficients solve M_1 x = r with the unweighted 2-form mass
//   (M_1)_ij = int_Omegahat vhat_i^T (J^T J / det J) vhat_j dxhat.
// Both integrals use the Gauss-Legendre rule with p_a + 1 points per element
// and axis, the rule of the Hodge masses.  The system is solved by conjugate
// gradients preconditioned with the identity-map mass, which is the Kronecker
// product of 1D masses per component and is solved exactly by banded sweeps:
// on the identity map the preconditioner is M_1 itself.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "setup.h"
#include "smx.h"

namespace smx {
namespace {

struct Axis1D {
    int q = 0;                 // Gauss points per element
    std::vector<double> x, w;  // on [0, 1]
};

// One component of the 2-form space: kinds and extents per axis.
struct Comp {
    int kind[3], deg[3], dim[3], off[3];
    long long base;
};

struct Space {
    int p[3], nel[3];
    Comp c[3];
    long long total;
    Axis1D ax[3];
    // basis values: per axis and kind, [element][point][r], r = 0..deg
    std::vector<double> bval[3][4];
};

void build_space(Space& S, const int p[3], const int nel[3], int field) {
    for (int a = 0; a < 3; ++a) {
        S.p[a] = p[a];
        S.nel[a] = nel[a];
        S.ax[a].q = p[a] + 1;
        gauss_legendre01(S.ax[a].q, S.ax[a].x, S.ax[a].w);
        for (int kind = 0; kind < 4; ++kind) {
            const int d = kind_degree(kind, p[a]);
            S.bval[a][kind].assign((size_t)nel[a] * S.ax[a].q * (d + 1), 0.0);
            for (int e = 0; e < nel[a]; ++e)
                for (int k = 0; k < S.ax[a].q; ++k) {
                    double v[16];
                    local_basis(kind, p[a], nel[a], e, (e + S.ax[a].x[k]) / nel[a], v);
                    for (int r = 0; r <= d; ++r) S.bval[a][kind][((size_t)e * S.ax[a].q + k) * (d + 1) + r] = v[r];
                }
        }
    }
    long long off = 0;
    for (int c = 0; c < 3; ++c) {
        Comp& C = S.c[c];
        long long n = 1;
        for (int a = 0; a < 3; ++a) {
            C.kind[a] = kFieldKinds[field][c][a];
            C.deg[a] = kind_degree(C.kind[a], p[a]);
            C.dim[a] = kind_dim(C.kind[a], p[a], nel[a]);
            C.off[a] = kind_offset(C.kind[a]);
            n *= C.dim[a];
        }
        C.base = off;
        off += n;
    }
    S.total = off;
}

// Visit every quadrature point of the element slab at z-element ez: for each
// point, its parametric position, weight (without det J) and element indices.
template <class F>
void for_slab_points(const Space& S, int ez, F&& f) {
    const int qx = S.ax[0].q, qy = S.ax[1].q, qz = S.ax[2].q;
    for (int kz = 0; kz < qz; ++kz)
        for (int ey = 0; ey < S.nel[1]; ++ey)
            for (int ky = 0; ky < qy; ++ky)
                for (int ex = 0; ex < S.nel[0]; ++ex)
                    for (int kx = 0; kx < qx; ++kx) {
                        const double xh[3] = {(ex + S.ax[0].x[kx]) / S.nel[0], (ey + S.ax[1].x[ky]) / S.nel[1],
                                              (ez + S.ax[2].x[kz]) / S.nel[2]};
                        const double w = S.ax[0].w[kx] / S.nel[0] * S.ax[1].w[ky] / S.nel[1] * S.ax[2].w[kz] / S.nel[2];
                        const int e[3] = {ex, ey, ez}, k[3] = {kx, ky, kz};
                        f(xh, w, e, k);
                    }
}

// The element's basis values per component and axis: (q x (deg + 1)) arrays.
void element_basis(const Space& S, const int e[3], const double* bas[3][3]) {
    for (int c = 0; c < 3; ++c)
        for (int ax = 0; ax < 3; ++ax)
            bas[c][ax] = &S.bval[ax][S.c[c].kind[ax]][(size_t)e[ax] * S.ax[ax].q * (S.c[c].deg[ax] + 1)];
}

// y += the integrals of U_c (values times weights at the element's q^3 points,
// component-major, x fastest) against the element's basis functions, by three
// 1D contractions (t1, t2: scratch of kRMax * 16 * 16 doubles).
void integrate_element(const Space& S, const int e[3], const double* const bas[3][3], const double* U,
                       std::vector<double>& y, double* t1, double* t2) {
    constexpr int R = kRMax;
    const int qx = S.ax[0].q, qy = S.ax[1].q, qz = S.ax[2].q, nq = qx * qy * qz;
    const int ex = e[0], ey = e[1], ez = e[2];
    for (int c = 0; c < 3; ++c) {
        const Comp& C = S.c[c];
        const int n0 = C.deg[0] + 1, n1 = C.deg[1] + 1, n2 = C.deg[2] + 1;
        for (int rz = 0; rz < n2; ++rz)
            for (int ky = 0; ky < qy; ++ky)
                for (int kx = 0; kx < qx; ++kx) {
                    double acc = 0.0;
                    for (int kz = 0; kz < qz; ++kz)
                        acc += bas[c][2][kz * n2 + rz] * U[(size_t)c * nq + (kz * qy + ky) * qx + kx];
                    t2[(rz * 16 + ky) * 16 + kx] = acc;
                }
        for (int rz = 0; rz < n2; ++rz)
            for (int ry = 0; ry < n1; ++ry)
                for (int kx = 0; kx < qx; ++kx) {
                    double acc = 0.0;
                    for (int ky = 0; ky < qy; ++ky) acc += bas[c][1][ky * n1 + ry] * t2[(rz * 16 + ky) * 16 + kx];
                    t1[(rz * R + ry) * 16 + kx] = acc;
                }
        for (int rz = 0; rz < n2; ++rz)
            for (int ry = 0; ry < n1; ++ry)
                for (int rx = 0; rx < n0; ++rx) {
                    const int ix = ex + rx + C.off[0], iy = ey + ry + C.off[1], iz = ez + rz + C.off[2];
                    if (ix < 0 || ix >= C.dim[0] || iy < 0 || iy >= C.dim[1] || iz < 0 || iz >= C.dim[2]) continue;
                    double acc = 0.0;
                    for (int kx = 0; kx < qx; ++kx) acc += bas[c][0][kx * n0 + rx] * t1[(rz * R + ry) * 16 + kx];
                    y[C.base + ix + (long long)C.dim[0] * (iy + (long long)C.dim[1] * iz)] += acc;
                }
    }
}

// y = M_1 x, matrix-free and element by element with sum factorisation: each
// component's local coefficients are interpolated to the element's q^3 points
// by three 1D contractions, multiplied by w J^T J / det J there, and
// integrated back by the transposed contractions.
// Gm: per quadrature point (slab order of for_slab_points, slabs along z in turn) the six
// entries 00 01 02 11 12 22 of w J^T J / det J.
void mass_apply(const Space& S, const std::vector<double>& Gm, const std::vector<double>& x, std::vector<double>& y) {
    std::fill(y.begin(), y.end(), 0.0);
    const int qx = S.ax[0].q, qy = S.ax[1].q, qz = S.ax[2].q, nq = qx * qy * qz;
    constexpr int R = kRMax;  // largest local count per axis (p + 1)
    std::vector<double> U(3 * (size_t)nq), loc((size_t)R * R * R), t1((size_t)R * R * 16), t2((size_t)R * 16 * 16);
    for (int ez = 0; ez < S.nel[2]; ++ez)
        for (int ey = 0; ey < S.nel[1]; ++ey)
            for (int ex = 0; ex < S.nel[0]; ++ex) {
                const int e[3] = {ex, ey, ez};
                const double* bas[3][3];  // [component][axis]
                element_basis(S, e, bas);
                // interpolate: loc[rz][ry][rx] -> U_c[kz][ky][kx]
                for (int c = 0; c < 3; ++c) {
                    const Comp& C = S.c[c];
                    const int n0 = C.deg[0] + 1, n1 = C.deg[1] + 1, n2 = C.deg[2] + 1;
                    for (int rz = 0; rz < n2; ++rz)
                        for (int ry = 0; ry < n1; ++ry)
                            for (int rx = 0; rx < n0; ++rx) {
                                const int ix = ex + rx + C.off[0], iy = ey + ry + C.off[1], iz = ez + rz + C.off[2];
                                const bool in = ix >= 0 && ix < C.dim[0] && iy >= 0 && iy < C.dim[1] && iz >= 0 &&
                                                iz < C.dim[2];
                                loc[(rz * R + ry) * R + rx] =
                                    in ? x[C.base + ix + (long long)C.dim[0] * (iy + (long long)C.dim[1] * iz)] : 0.0;
                            }
                    for (int rz = 0; rz < n2; ++rz)
                        for (int ry = 0; ry < n1; ++ry)
                            for (int kx = 0; kx < qx; ++kx) {
                                double acc = 0.0;
                                for (int rx = 0; rx < n0; ++rx) acc += bas[c][0][kx * n0 + rx] * loc[(rz * R + ry) * R + rx];
                                t1[(rz * R + ry) * 16 + kx] = acc;
                            }
                    for (int rz = 0; rz < n2; ++rz)
                        for (int ky = 0; ky < qy; ++ky)
                            for (int kx = 0; kx < qx; ++kx) {
                                double acc = 0.0;
                                for (int ry = 0; ry < n1; ++ry) acc += bas[c][1][ky * n1 + ry] * t1[(rz * R + ry) * 16 + kx];
                                t2[(rz * 16 + ky) * 16 + kx] = acc;
                            }
                    for (int kz = 0; kz < qz; ++kz)
                        for (int ky = 0; ky < qy; ++ky)
                            for (int kx = 0; kx < qx; ++kx) {
                                double acc = 0.0;
                                for (int rz = 0; rz < n2; ++rz) acc += bas[c][2][kz * n2 + rz] * t2[(rz * 16 + ky) * 16 + kx];
                                U[(size_t)c * nq + (kz * qy + ky) * qx + kx] = acc;
                            }
                }
                // the metric at every point of the element
                const long long slab = (long long)S.nel[0] * qx * S.nel[1] * qy * qz;
                for (int kz = 0; kz < qz; ++kz)
                    for (int ky = 0; ky < qy; ++ky)
                        for (int kx = 0; kx < qx; ++kx) {
                            const long long pt = ez * slab + (((long long)kz * S.nel[1] + ey) * qy + ky) *
                                                                 ((long long)S.nel[0] * qx) + ex * qx + kx;
                            const double* g = &Gm[6 * pt];
                            const size_t qi = (size_t)(kz * qy + ky) * qx + kx;
                            const double u[3] = {U[qi], U[nq + qi], U[2 * (size_t)nq + qi]};
                            U[qi] = g[0] * u[0] + g[1] * u[1] + g[2] * u[2];  // u was copied: overwrite in place
                            U[nq + qi] = g[1] * u[0] + g[3] * u[1] + g[4] * u[2];
                            U[2 * (size_t)nq + qi] = g[2] * u[0] + g[4] * u[1] + g[5] * u[2];
                        }
                integrate_element(S, e, bas, U.data(), y, t1.data(), t2.data());
            }
}

// The identity-map mass: per component the Kronecker product of the 1D masses
// of its kinds; its inverse by banded sweeps along x, y and z.
struct KronMass {
    BandLU f[3][3];  // [component][axis]
};

bool build_kron(const Space& S, KronMass& K) {
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a) {
            const Comp& C = S.c[c];
            const int n = C.dim[a], d = C.deg[a];
            std::vector<double> M((size_t)n * n, 0.0);
            for (int e = 0; e < S.nel[a]; ++e) {
                const std::vector<double> Me = element_mass(C.kind[a], S.p[a], S.nel[a], e);
                for (int r = 0; r <= d; ++r)
                    for (int t = 0; t <= d; ++t) {
                        const int i = e + r + C.off[a], j = e + t + C.off[a];
                        if (i >= 0 && i < n && j >= 0 && j < n) M[(size_t)i * n + j] += Me[r * (d + 1) + t];
                    }
            }
            if (!band_lu(M, n, d, d, K.f[c][a])) return false;
        }
    return true;
}

void band_solve(const BandLU& F, double* v, long long stride) {
    const int n = F.n;
    for (int m = 0; m < n; ++m) {
        double u = v[m * stride];
        for (int k = 1; k <= F.kl && k <= m; ++k) u -= F.L[m * F.kl + k - 1] * v[(m - k) * stride];
        v[m * stride] = u;
    }
    for (int m = n - 1; m >= 0; --m) {
        double u = v[m * stride] * F.dinv[m];
        for (int k = 1; k <= F.ku && m + k < n; ++k) u -= F.U[m * F.ku + k - 1] * v[(m + k) * stride];
        v[m * stride] = u;
    }
}

void kron_solve(const Space& S, const KronMass& K, std::vector<double>& v) {
    for (int c = 0; c < 3; ++c) {
        const Comp& C = S.c[c];
        const long long nx = C.dim[0], ny = C.dim[1], nz = C.dim[2];
        double* base = v.data() + C.base;
        for (long long k = 0; k < nz; ++k)
            for (long long j = 0; j < ny; ++j) band_solve(K.f[c][0], base + nx * (j + ny * k), 1);
        for (long long k = 0; k < nz; ++k)
            for (long long i = 0; i < nx; ++i) band_solve(K.f[c][1], base + i + nx * ny * k, nx);
        for (long long j = 0; j < ny; ++j)
            for (long long i = 0; i < nx; ++i) band_solve(K.f[c][2], base + i + nx * j, nx * ny);
    }
}

double dot(const std::vector<double>& a, const std::vector<double>& b) {
    double s = 0.0;
    for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
    return s;
}

}  // namespace

int l2_project_2form(const int p[3], const int nel[3], const GeomMap& geom, int field, project_fn fn, void* user,
                     double* out, double rtol, int maxit, int* iters) {
    Space S;
    build_space(S, p, nel, field);
    const long long N = S.total;
    // right-hand side, one callback (and one geometry evaluation) per slab of elements along z;
    // the metric w J^T J / det J of every point is kept for the mass applies
    const long long slab_pts = (long long)S.nel[0] * S.ax[0].q * S.nel[1] * S.ax[1].q * S.ax[2].q;
    std::vector<double> Gm(6 * slab_pts * S.nel[2]);
    std::vector<double> r(N, 0.0), X3, V3, XH, J3;
    std::vector<double> U(3 * (size_t)S.ax[0].q * S.ax[1].q * S.ax[2].q), t1((size_t)kRMax * kRMax * 16),
        t2((size_t)kRMax * 16 * 16);
    for (int ez = 0; ez < S.nel[2]; ++ez) {
        XH.clear();
        for_slab_points(S, ez, [&](const double* xh, double, const int*, const int*) { XH.insert(XH.end(), xh, xh + 3); });
        const long long n = (long long)XH.size() / 3;
        X3.assign(3 * n, 0.0);
        J3.assign(9 * n, 0.0);
        const int gst = geometry_eval_points(geom, n, XH.data(), X3.data(), J3.data());
        if (gst) return gst;
        {
            long long pt = 0;
            for_slab_points(S, ez, [&](const double*, double w, const int*, const int*) {
                const double* J = &J3[9 * pt];
                const double sc = w / det3(J);
                double* g = &Gm[6 * (ez * slab_pts + pt)];
                const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
                for (int k = 0; k < 6; ++k) {
                    const int i = ij[k][0], j = ij[k][1];
                    g[k] = sc * (J[i] * J[j] + J[3 + i] * J[3 + j] + J[6 + i] * J[6 + j]);
                }
                ++pt;
            });
        }
        V3.assign(3 * n, 0.0);
        fn(n, X3.data(), V3.data(), user);
        for (long long i = 0; i < 3 * n; ++i)
            if (!std::isfinite(V3[i])) return SMX_ENONFINITE;
        // slab point (ex, kx, ey, ky, kz) sits at ((kz nel_y + ey) q_y + ky) nel_x q_x + ex q_x + kx
        const int qx = S.ax[0].q, qy = S.ax[1].q, qz = S.ax[2].q, nq = qx * qy * qz;
        for (int ey = 0; ey < S.nel[1]; ++ey)
            for (int ex = 0; ex < S.nel[0]; ++ex) {
                const int e[3] = {ex, ey, ez};
                for (int kz = 0; kz < qz; ++kz)
                    for (int ky = 0; ky < qy; ++ky)
                        for (int kx = 0; kx < qx; ++kx) {
                            const double w = S.ax[0].w[kx] / S.nel[0] * S.ax[1].w[ky] / S.nel[1] * S.ax[2].w[kz] /
                                             S.nel[2];
                            const long long pt =
                                (((long long)kz * S.nel[1] + ey) * qy + ky) * ((long long)S.nel[0] * qx) + ex * qx + kx;
                            const double* J = &J3[9 * pt];
                            const double* V = &V3[3 * pt];
                            const size_t qi = (size_t)(kz * qy + ky) * qx + kx;
                            for (int c = 0; c < 3; ++c)  // w (J^T V)_c
                                U[(size_t)c * nq + qi] = w * (J[c] * V[0] + J[3 + c] * V[1] + J[6 + c] * V[2]);
                        }
                const double* bas[3][3];
                element_basis(S, e, bas);
                integrate_element(S, e, bas, U.data(), r, t1.data(), t2.data());
            }
    }
    KronMass K;
    if (!build_kron(S, K)) return SMX_ESINGULAR;
    // preconditioned conjugate gradients from x = P^{-1} r
    std::vector<double> x = r, res(N), z(N), d(N), Ad(N);
    kron_solve(S, K, x);
    mass_apply(S, Gm, x, Ad);
    for (long long i = 0; i < N; ++i) res[i] = r[i] - Ad[i];
    const double rnorm0 = std::sqrt(dot(r, r));
    int it = 0;
    if (rnorm0 > 0.0 && std::sqrt(dot(res, res)) > rtol * rnorm0) {
        z = res;
        kron_solve(S, K, z);
        d = z;
        double rz = dot(res, z);
        for (it = 1; it <= maxit; ++it) {
            mass_apply(S, Gm, d, Ad);
            const double alpha = rz / dot(d, Ad);
            for (long long i = 0; i < N; ++i) {
                x[i] += alpha * d[i];
                res[i] -= alpha * Ad[i];
            }
            if (std::sqrt(dot(res, res)) <= rtol * rnorm0) break;
            z = res;
            kron_solve(S, K, z);
            const double rz1 = dot(res, z);
            const double beta = rz1 / rz;
            rz = rz1;
            for (long long i = 0; i < N; ++i) d[i] = z[i] + beta * d[i];
        }
        if (it > maxit) return SMX_ESINGULAR;
    }
    if (iters) *iters = it;
    std::copy(x.begin(), x.end(), out);
    return SMX_OK;
}

}  // namespace smx
