// C ABI of the scheme-2 leapfrog (include/smx.h): host setup, workspace
// binding and the enqueue of the device kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/smx.h"
#include "internal.h"
#include "setup.h"

#include <atomic>

using namespace smx;

namespace smx {
int noalloc_region(void** base, uint64_t** owner);  // noalloc.cu
}

namespace {

struct HodgeHost {
    int mode = 0;  // 0 block Kronecker, 1 quadrature
    // identity map and constant material: the mass is one Kronecker product of
    // 1D masses, lmass[a][kind] (n x (2 deg + 1) band rows, material folded into axis x)
    bool separable = false;
    std::vector<double> lmass[3][4];
    size_t o_lmass[3][4];
    // block mode
    int ntile[3] = {0, 0, 0};
    int max_nloc = 0;
    std::vector<int> tf0[3], tlen[3];
    std::vector<double> tmat[3];
    std::vector<double> gamma;
    std::vector<int> tile_block;  // block material: the block of each tile
    // quadrature mode
    int q[3] = {0, 0, 0};
    std::vector<double> bval[3];
    std::vector<double> G;
    long long Qtot = 0;
    int Qn[3] = {0, 0, 0};
    // device offsets in the workspace (bytes)
    size_t o_tf0[3] = {}, o_tlen[3] = {}, o_tmat[3] = {}, o_gamma = 0, o_bval[3] = {}, o_G = 0;
};

struct Blob {
    std::vector<unsigned char> bytes;
    template <class T>
    size_t add(const std::vector<T>& v) {
        const size_t off = (bytes.size() + 255) & ~size_t(255);
        bytes.resize(off + v.size() * sizeof(T));
        if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
        return off;
    }
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    const void* key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double dt = 0.0;
    int nsteps = 0;
    long long kernels = 0;  // kernel nodes per replay
};

// Context ids: the static no-alloc array records which id's tables it holds, so a
// context whose tables change takes a fresh id and the next no-alloc call re-uploads.
std::atomic<uint64_t> g_next_uid{1};

uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

struct smx_ctx {
    uint64_t uid = 0;  // unique per context (which tables the static no-alloc array holds)
    int p[3], nel[3];
    int geometry;
    double amp;
    GeomMap gmap;  // the map F (built-in or host callback)
    DevField fld[4];
    long long N_e, N_h;
    BandLU fac[3][4];  // per axis: G, M, G^T, M^T
    HodgeHost hodge[2];  // 0: B (mu), 1: D (eps)
    Blob blob;
    size_t o_fac[3][4][3];
    size_t tables_bytes = 0, o_scratch = 0, o_scratch2 = 0, o_partial = 0, o_dots = 0, total_bytes = 0;
    unsigned char* ws = nullptr;
    cudaStream_t stream = nullptr;
    // device argument blocks (valid once bound)
    SolveArgs solve[2][3];  // [K1, Kt1][axis]
    HodgeBlockArgs hb[2];
    HodgeQuadArgs hq[2];
    MassSolveArgs ms[2][3];  // separable Hodge star: [field][axis]
    double* scratch = nullptr;
    double* scratch2 = nullptr;
    double* state = nullptr;  // d, e (N_e each), b, h (N_h each) for smx_step_host
    size_t o_state = 0;
    long long launches = 0;
    int timing = 0;
    struct Timed {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Timed> timed;
    double* partial = nullptr;
    double* dots = nullptr;
    // mixed precision: FP32 (hi, lo) tables, FP32 intermediates e32, h32, y32
    int precision = SMX_FP64;
    size_t o_fac32[3][4][3];
    size_t o_tmat32[2][3], o_lmass32[2][3][4];
    size_t o_e32 = 0, o_h32 = 0, o_y32 = 0;
    float *e32 = nullptr, *h32 = nullptr, *y32 = nullptr;
    HodgeBlockF32Args hb32[2];
    size_t o_bval32[2][3], o_G32[2];  // quadrature Hodge (curved map / pointwise material): FP32 tables
    HodgeQuadF32Args hq32[2];
    LineF32Args ln32[2][3];  // [field][axis]: plain pairing sweeps (block Hodge) or fused mass + solve (separable)
    // captured CUDA graph of the last smx_step call, keyed by its pointers, dt and nsteps
    int use_graphs = 1;
    GraphCache graph;
    bool use_mode = false;   // dense mode products instead of line recurrences (every line length <= kModeMaxN)
    size_t o_mode32[2][3][3];
    ModeF32Args md32[2][3];  // [field][axis]
    // the same operators as three BF16 parts for the tensor-core kernel (the default)
    int mode_kernel = SMX_MODE_AUTO;
    // FP64 context: the same dense operators as digit planes for the FP64 tensor-core
    // mode products (every line length <= kModeMaxN); mode_kernel then selects them
    bool use_digit = false;
    size_t o_dig[2][3][3], o_dige[2][3][3];
    ModeDigitArgs mdg[2][3];  // [field][axis]
    size_t o_status = 0;          // device status word (bit 0: a tensor-core wait gave up)
    unsigned* status = nullptr;
    // reverse step: transposed pairing sweeps, block permittivity, receivers
    SolveArgs solveT[2][3];       // [K_1^T, K~_1^T][axis]
    bool eps_blocks = false;      // eps given on a block grid: gradients and updates available
    int eps_nb[3] = {0, 0, 0}, eps_epb[3] = {0, 0, 0};
    std::vector<double> eps_vals;  // current block values (x fastest)
    size_t o_pair_scale = 0, o_tile_block = 0;
    PairArgs pair{};
    std::vector<int> rec_ptr, rec_idx;
    std::vector<double> rec_val;
    size_t o_rec_ptr = 0, o_rec_idx = 0, o_rec_val = 0;
    RecArgs rec{};
    // refined mixed step: band rows of the 1D pairing factors (G, M, G^T, M^T per axis) for the
    // FP64 residual, a second FP64 vector, and the residual passes [field][axis]
    std::vector<double> band_rows[3][4];
    size_t o_band[3][4] = {};
    // scheme 1 (mass-matrix Hodge stars): 1-form masses [0] M~^1_mu (field H), [1] M^1_eps (field E),
    // the unit-material Kronecker masses of every kind per axis as the PCG preconditioner (banded LU
    // with half-bandwidth p), three PCG vectors and the PCG scalars, and the argument blocks
    bool s1 = false;
    HodgeHost hodge1[2];
    BandLU mfac[3][4];
    size_t o_mfac[3][4][3] = {};
    size_t o_s1v[3] = {}, o_cg = 0;
    double* s1v[3] = {nullptr, nullptr, nullptr};
    double* cg = nullptr;
    HodgeBlockArgs hb1[2];
    HodgeQuadArgs hq1[2];
    SolveArgs pre1[2][3];
    BandApplyArgs kt[2][3];  // [0] K_2 = K~_1^T (B -> H layout), [1] K~_2 = K_1^T (D -> E layout)
    size_t o_t64 = 0;
    double* t64 = nullptr;
    BandApplyArgs band[2][3];
    // refined reverse step: FP32 sweeps and FP64 residual passes with the transposed 1D factors,
    // [which][axis] with which = 0 for K_1^T (D layout), 1 for K~_1^T (B layout)
    LineF32Args ln32T[2][3];
    BandApplyArgs bandT[2][3];
};

namespace {

const int kFieldOfHodge[2] = {SMX_FIELD_B, SMX_FIELD_D};

// Host twin of the device metric rescale: every quadrature point's six metric
// entries in the blob times ratio[block of its element], and the mixed form's
// (hi, lo) copy rebuilt from the product.
void rescale_metric_host(smx_ctx* C, const std::vector<double>& ratio) {
    const HodgeHost& H = C->hodge[1];
    const long long Q = H.Qtot;
    double* G = reinterpret_cast<double*>(C->blob.bytes.data() + H.o_G);
    float* G32 = C->precision != SMX_FP64 ? reinterpret_cast<float*>(C->blob.bytes.data() + C->o_G32[1]) : nullptr;
    for (long long i = 0; i < Q; ++i) {
        const long long qx = i % H.Qn[0], r = i / H.Qn[0], qy = r % H.Qn[1], qz = r / H.Qn[1];
        const int bx = (int)(qx / H.q[0]) / C->eps_epb[0], by = (int)(qy / H.q[1]) / C->eps_epb[1];
        const int bz = (int)(qz / H.q[2]) / C->eps_epb[2];
        const double f = ratio[((size_t)bz * C->eps_nb[1] + by) * C->eps_nb[0] + bx];
        for (int k = 0; k < 6; ++k) {
            const double v = f * G[k * Q + i];
            G[k * Q + i] = v;
            if (G32) {
                const float hi = static_cast<float>(v);
                G32[2 * (k * Q + i)] = hi;
                G32[2 * (k * Q + i) + 1] = static_cast<float>(v - static_cast<double>(hi));
            }
        }
    }
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int check_material(const smx_material& m, const int nel[3]) {
    if (m.kind == SMX_MAT_CONST) return finite_pos(m.value) ? SMX_OK : SMX_EMAT;
    if (m.kind == SMX_MAT_BLOCKS) {
        if (!m.block_values) return SMX_EINVAL;
        for (int a = 0; a < 3; ++a)
            if (m.blocks[a] < 1 || nel[a] % m.blocks[a] != 0) return SMX_EINVAL;
        const long long nb = (long long)m.blocks[0] * m.blocks[1] * m.blocks[2];
        for (long long i = 0; i < nb; ++i)
            if (!finite_pos(m.block_values[i])) return SMX_EMAT;
        return SMX_OK;
    }
    if (m.kind == SMX_MAT_POINTWISE) return m.fn ? SMX_OK : SMX_EINVAL;
    return SMX_EINVAL;
}

// Element ranges of the Hodge tiles along one axis: every material block is cut
// into ceil(len/8) nearly equal tiles so no tile straddles a material jump.
std::vector<int> tile_bounds(int nel, int nblocks) {
    std::vector<int> b{0};
    const int bl = nel / nblocks;
    for (int k = 0; k < nblocks; ++k) {
        const int lo = k * bl, nt = (bl + kTileMax - 1) / kTileMax;
        for (int t = 1; t <= nt; ++t) b.push_back(lo + (int)((long long)bl * t / nt));
    }
    return b;
}

// Block-Kronecker tables of the mass of `field` with weight 1/material (invert, the 2-form
// masses of scheme 2) or the material itself (the 1-form masses of scheme 1).
int build_hodge_block_t(smx_ctx* C, HodgeHost& H, int field, const smx_material& m, bool invert) {
    std::vector<int> bounds[3];
    for (int a = 0; a < 3; ++a) {
        const int nb = (m.kind == SMX_MAT_BLOCKS) ? m.blocks[a] : 1;
        bounds[a] = tile_bounds(C->nel[a], nb);
        H.ntile[a] = (int)bounds[a].size() - 1;
    }
    for (int a = 0; a < 3; ++a) {
        const int p = C->p[a], nel = C->nel[a], nt = H.ntile[a];
        H.tf0[a].assign(4 * nt, 0);
        H.tlen[a].assign(4 * nt, 0);
        H.tmat[a].assign((size_t)4 * nt * kLMax * kLMax, 0.0);
        for (int kind = 0; kind < 4; ++kind) {
            const int d = kind_degree(kind, p), off = kind_offset(kind), dim = kind_dim(kind, p, nel);
            for (int t = 0; t < nt; ++t) {
                const int e0 = bounds[a][t], e1 = bounds[a][t + 1];
                const int flo = std::max(0, e0 + off), fhi = std::min(dim - 1, e1 - 1 + d + off);
                const int len = fhi - flo + 1;
                if (len > kLMax || len < 1) return SMX_EINVAL;
                H.tf0[a][kind * nt + t] = flo;
                H.tlen[a][kind * nt + t] = len;
                double* M = &H.tmat[a][(size_t)(kind * nt + t) * kLMax * kLMax];
                for (int e = e0; e < e1; ++e) {
                    const std::vector<double> Me = element_mass(kind, p, nel, e);
                    for (int r = 0; r <= d; ++r) {
                        const int i = e + r + off;
                        if (i < 0 || i >= dim) continue;
                        for (int s = 0; s <= d; ++s) {
                            const int j = e + s + off;
                            if (j < 0 || j >= dim) continue;
                            M[(i - flo) * kLMax + (j - flo)] += Me[r * (d + 1) + s];
                        }
                    }
                }
            }
        }
    }
    H.max_nloc = 0;
    for (int c = 0; c < 3; ++c) {
        int lmax[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) {
            const int kind = kFieldKinds[field][c][a];
            for (int t = 0; t < H.ntile[a]; ++t) lmax[a] = std::max(lmax[a], H.tlen[a][kind * H.ntile[a] + t]);
        }
        H.max_nloc = std::max(H.max_nloc, lmax[0] * lmax[1] * lmax[2]);
    }
    H.gamma.assign((size_t)H.ntile[0] * H.ntile[1] * H.ntile[2], 0.0);
    for (int tz = 0; tz < H.ntile[2]; ++tz)
        for (int ty = 0; ty < H.ntile[1]; ++ty)
            for (int tx = 0; tx < H.ntile[0]; ++tx) {
                double v = m.value;
                if (m.kind == SMX_MAT_BLOCKS) {
                    const int t3[3] = {tx, ty, tz};
                    int b3[3];
                    for (int a = 0; a < 3; ++a) b3[a] = bounds[a][t3[a]] / (C->nel[a] / m.blocks[a]);
                    const int blk = (b3[2] * m.blocks[1] + b3[1]) * m.blocks[0] + b3[0];
                    v = m.block_values[blk];
                    H.tile_block.push_back(blk);
                }
                H.gamma[((size_t)tz * H.ntile[1] + ty) * H.ntile[0] + tx] = invert ? 1.0 / v : v;
            }
    return SMX_OK;
}

int build_hodge_block(smx_ctx* C, int h, const smx_material& m) {
    return build_hodge_block_t(C, C->hodge[h], kFieldOfHodge[h], m, true);
}

// Global univariate masses of every space kind as band rows (half-bandwidth =
// the kind's degree), gamma folded into the x axis: M = gamma Mz (x) My (x) Mx.
void build_separable(smx_ctx* C, int h, double gamma) {
    HodgeHost& H = C->hodge[h];
    H.separable = true;
    for (int a = 0; a < 3; ++a) {
        const int p = C->p[a], nel = C->nel[a];
        for (int kind = 0; kind < 4; ++kind) {
            const int d = kind_degree(kind, p), off = kind_offset(kind), dim = kind_dim(kind, p, nel);
            const int W = 2 * d + 1;
            std::vector<double>& R = H.lmass[a][kind];
            R.assign((size_t)dim * W, 0.0);
            const double scale = a == 0 ? gamma : 1.0;
            for (int e = 0; e < nel; ++e) {
                const std::vector<double> Me = element_mass(kind, p, nel, e);
                for (int r = 0; r <= d; ++r) {
                    const int i = e + r + off;
                    if (i < 0 || i >= dim) continue;
                    for (int s = 0; s <= d; ++s) {
                        const int j = e + s + off;
                        if (j < 0 || j >= dim) continue;
                        R[(size_t)i * W + (j - i + d)] += scale * Me[r * (d + 1) + s];
                    }
                }
            }
        }
    }
}

// Quadrature tables: basis values and, per point, the metric of a 2-form mass weighted by
// 1/material, w J^T J / (det J material) (one_form = false), or of a 1-form mass weighted by the
// material, w material det J (J^T J)^{-1} (one_form = true: u = J^{-T} u^, Sec. 2.3).
int build_hodge_quad_t(smx_ctx* C, HodgeHost& H, const smx_material& m, bool one_form) {
    std::vector<double> gx[3], gw[3];
    for (int a = 0; a < 3; ++a) {
        const int p = C->p[a], nel = C->nel[a];
        H.q[a] = p + 1;
        H.Qn[a] = nel * H.q[a];
        gauss_legendre01(H.q[a], gx[a], gw[a]);
        H.bval[a].assign((size_t)4 * nel * H.q[a] * kRMax, 0.0);
        for (int kind = 0; kind < 4; ++kind)
            for (int e = 0; e < nel; ++e)
                for (int k = 0; k < H.q[a]; ++k) {
                    double v[16];
                    local_basis(kind, p, nel, e, (e + gx[a][k]) / nel, v);
                    const int d = kind_degree(kind, p);
                    for (int r = 0; r <= d; ++r)
                        H.bval[a][(((size_t)kind * nel + e) * H.q[a] + k) * kRMax + r] = v[r];
                }
    }
    H.Qtot = (long long)H.Qn[0] * H.Qn[1] * H.Qn[2];
    const long long Q = H.Qtot;
    std::vector<double> X3(3 * Q), Jall(9 * Q), wdet(Q);
    {
        std::vector<double> xh(3 * Q);
        for (long long qi = 0; qi < Q; ++qi) {
            const int ii[3] = {(int)(qi % H.Qn[0]), (int)((qi / H.Qn[0]) % H.Qn[1]),
                               (int)(qi / ((long long)H.Qn[0] * H.Qn[1]))};
            double w = 1.0;
            for (int a = 0; a < 3; ++a) {
                const int e = ii[a] / H.q[a], k = ii[a] % H.q[a];
                xh[3 * qi + a] = (e + gx[a][k]) / C->nel[a];
                w *= gw[a][k] / C->nel[a];
            }
            wdet[qi] = w;
        }
        // F and J_F at every quadrature point (one callback call for a host map); det J_F > 0 checked
        const int st = geometry_eval_points(C->gmap, Q, xh.data(), X3.data(), Jall.data());
        if (st) return st;
        for (long long qi = 0; qi < Q; ++qi) wdet[qi] /= det3(&Jall[9 * qi]);
    }
    std::vector<double> mat(Q);
    if (m.kind == SMX_MAT_POINTWISE) {
        m.fn(Q, X3.data(), mat.data(), m.user);
    } else {
        for (long long qi = 0; qi < Q; ++qi) {
            double v = m.value;
            if (m.kind == SMX_MAT_BLOCKS) {
                const int ix = (int)(qi % H.Qn[0]);
                const int iy = (int)((qi / H.Qn[0]) % H.Qn[1]);
                const int iz = (int)(qi / ((long long)H.Qn[0] * H.Qn[1]));
                const int ii[3] = {ix, iy, iz};
                int b3[3];
                for (int a = 0; a < 3; ++a) b3[a] = (ii[a] / H.q[a]) / (C->nel[a] / m.blocks[a]);
                v = m.block_values[(b3[2] * m.blocks[1] + b3[1]) * m.blocks[0] + b3[0]];
            }
            mat[qi] = v;
        }
    }
    H.G.assign(6 * Q, 0.0);
    for (long long qi = 0; qi < Q; ++qi) {
        if (!finite_pos(mat[qi])) return SMX_EMAT;
        const double* J = &Jall[9 * qi];
        double JtJ[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) JtJ[i][j] = J[i] * J[j] + J[3 + i] * J[3 + j] + J[6 + i] * J[6 + j];
        double s = wdet[qi] / mat[qi];
        if (one_form) {
            // (J^T J)^{-1} by cofactors; w det J material = (w / det J) det J^2 material
            const double dj = det3(J);
            double A[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) A[i][j] = JtJ[i][j];
            const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1], c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
            const double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0], c11 = A[0][0] * A[2][2] - A[0][2] * A[2][0];
            const double c12 = A[0][2] * A[1][0] - A[0][0] * A[1][2], c22 = A[0][0] * A[1][1] - A[0][1] * A[1][0];
            const double detA = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
            JtJ[0][0] = c00 / detA;
            JtJ[0][1] = JtJ[1][0] = c01 / detA;
            JtJ[0][2] = JtJ[2][0] = c02 / detA;
            JtJ[1][1] = c11 / detA;
            JtJ[1][2] = JtJ[2][1] = c12 / detA;
            JtJ[2][2] = c22 / detA;
            s = wdet[qi] * dj * dj * mat[qi];
        }
        H.G[0 * Q + qi] = s * JtJ[0][0];
        H.G[1 * Q + qi] = s * JtJ[0][1];
        H.G[2 * Q + qi] = s * JtJ[0][2];
        H.G[3 * Q + qi] = s * JtJ[1][1];
        H.G[4 * Q + qi] = s * JtJ[1][2];
        H.G[5 * Q + qi] = s * JtJ[2][2];
    }
    return SMX_OK;
}

int build_hodge_quad(smx_ctx* C, int h, const smx_material& m) { return build_hodge_quad_t(C, C->hodge[h], m, false); }

// Dense A^{-1} (row-major) from a banded LU, column by column.
std::vector<double> dense_inverse(const BandLU& f) {
    const int n = f.n;
    std::vector<double> inv((size_t)n * n, 0.0), col(n);
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) col[i] = (i == j) ? 1.0 : 0.0;
        for (int m = 0; m < n; ++m)
            for (int k = 1; k <= f.kl; ++k)
                if (m - k >= 0) col[m] -= f.L[(size_t)m * f.kl + k - 1] * col[m - k];
        for (int m = n - 1; m >= 0; --m) {
            double v = col[m] * f.dinv[m];
            for (int k = 1; k <= f.ku; ++k)
                if (m + k < n) v -= f.U[(size_t)m * f.ku + k - 1] * col[m + k];
            col[m] = v;
        }
        for (int i = 0; i < n; ++i) inv[(size_t)i * n + j] = col[i];
    }
    return inv;
}

// Dense (n x n) product of a dense matrix with a banded one given as band rows (half-bandwidth d).
std::vector<double> dense_times_band(const std::vector<double>& A, const std::vector<double>& rows, int n, int d) {
    const int W = 2 * d + 1;
    std::vector<double> out((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const double a = A[(size_t)i * n + k];
            if (a == 0.0) continue;
            for (int q = 0; q < W; ++q) {
                const int j = k - d + q;
                if (j >= 0 && j < n) out[(size_t)i * n + j] += a * rows[(size_t)k * W + q];
            }
        }
    return out;
}

// FP64 values as FP32 (hi, lo) pairs: hi = fl32(v), lo = fl32(v - hi); hi + lo = v to about 2^-48 relative.
std::vector<float> split_pairs(const std::vector<double>& v) {
    std::vector<float> out(2 * v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        const float hi = static_cast<float>(v[i]);
        out[2 * i] = hi;
        out[2 * i + 1] = static_cast<float>(v[i] - static_cast<double>(hi));
    }
    return out;
}

std::vector<double> transpose(const std::vector<double>& A, int n) {
    std::vector<double> T(A.size());
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) T[(size_t)j * n + i] = A[(size_t)i * n + j];
    return T;
}

bool is_banded(const std::vector<double>& A, int n, int bw) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (std::abs(i - j) > bw && A[(size_t)i * n + j] != 0.0) return false;
    return true;
}

// Which 1D factor block c of K_1 (K1 = 0) or K~_1 (1) uses along axis a:
// (D1 rows, P0 cols) -> G, (D0, P1) -> M, transposed for K~_1 (Eq. tensor_K, Eq. tensor_Ktilde).
int factor_index(int which, int c, int a) {
    const int row_kind = kFieldKinds[which == 0 ? SMX_FIELD_D : SMX_FIELD_B][c][a];
    if (which == 0) return row_kind == D1 ? 0 : 1;
    return row_kind == P0 ? 2 : 3;
}

// Workspace layout: the tables (blob), then scratch, reduction, status,
// state and (mixed form) FP32 vectors, each 256-byte aligned.
void layout(smx_ctx* C) {
    C->tables_bytes = (C->blob.bytes.size() + 255) & ~size_t(255);
    C->o_scratch = C->tables_bytes;
    const size_t nmax = (size_t)std::max(C->N_e, C->N_h);
    C->o_scratch2 = C->o_scratch + ((nmax * sizeof(double) + 255) & ~size_t(255));
    C->o_partial = C->o_scratch2 + ((nmax * sizeof(double) + 255) & ~size_t(255));
    C->o_dots = C->o_partial + ((kDotBlocks * sizeof(double) + 255) & ~size_t(255));
    C->o_status = C->o_dots + 256;
    C->o_state = C->o_status + 256;
    C->total_bytes = C->o_state + ((2 * (size_t)(C->N_e + C->N_h) * sizeof(double) + 255) & ~size_t(255));
    if (C->precision != SMX_FP64) {
        auto f32 = [](long long n) { return ((size_t)n * sizeof(float) + 255) & ~size_t(255); };
        C->o_e32 = C->total_bytes;
        C->o_h32 = C->o_e32 + f32(C->N_e);
        C->o_y32 = C->o_h32 + f32(C->N_h);
        C->total_bytes = C->o_y32 + f32((long long)nmax);
    }
    if (C->s1) {  // PCG vectors and scalars of scheme 1
        for (int k = 0; k < 3; ++k) {
            C->o_s1v[k] = C->total_bytes;
            C->total_bytes += (nmax * sizeof(double) + 255) & ~size_t(255);
        }
        C->o_cg = C->total_bytes;
        C->total_bytes += 256;
    }
    if (C->precision == SMX_MIXED_REFINED) {  // a second FP64 vector for the residual passes
        C->o_t64 = C->total_bytes;
        C->total_bytes = C->o_t64 + ((nmax * sizeof(double) + 255) & ~size_t(255));
    }
}

#define CK(call)                                          \
    do {                                                  \
        cudaError_t err_ = (call);                        \
        if (err_ != cudaSuccess) return SMX_ECUDA;        \
    } while (0)

// Launch through f() and account for it: kernel count, and CUDA events around
// it when timing is on (class cls, see smx_kernel_times).
template <class F>
int run(smx_ctx* C, int cls, int nkernels, F&& f) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (C->timing) {
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        CK(cudaEventRecord(a, C->stream));
    }
    CK(f());
    if (C->timing) {
        CK(cudaEventRecord(b, C->stream));
        C->timed.push_back({cls, a, b});
    }
    C->launches += nkernels;
    return SMX_OK;
}

// zero (optional): the curl also clears this vector over its output range, so the
// Hodge apply that follows (accumulating into it) needs no zeroing launch.
int curl_primal_impl(smx_ctx* C, const double* e, double* b, double alpha, double* zero = nullptr) {
    return run(C, 0, 1, [&] {
        return launch_curl_primal(C->fld[SMX_FIELD_E], C->fld[SMX_FIELD_B], e, b, alpha, C->stream, zero);
    });
}

int curl_dual_impl(smx_ctx* C, const double* h, double* d, double alpha, const double* jhat, const double* amp,
                   int idx, double s, double* zero = nullptr) {
    return run(C, 1, 1, [&] {
        return launch_curl_dual(C->fld[SMX_FIELD_H], C->fld[SMX_FIELD_D], h, d, alpha, jhat, amp, idx, s, C->stream,
                                zero);
    });
}

// y = M x; prezeroed: y is already zero (cleared by the preceding curl)
int hodge_apply_impl(smx_ctx* C, int h, const double* x, double* y, bool prezeroed = false) {
    const DevField& F = C->fld[kFieldOfHodge[h]];
    if (!prezeroed) {
        const int st = run(C, 20, 1, [&] { return launch_zero(y, F.total, C->stream); });
        if (st) return st;
    }
    if (C->hodge[h].mode == 0) return run(C, 2, 1, [&] { return launch_hodge_block(C->hb[h], x, y, C->stream); });
    return run(C, 3, 1, [&] { return launch_hodge_quad(C->hq[h], x, y, C->stream); });
}

int solve_impl(smx_ctx* C, int which, const double* y, double* x) {
    // x-sweep reads y and writes x; the y and z sweeps work in place in x
    int st = run(C, 4, 1, [&] { return launch_solve_axis(C->solve[which][0], C->p[0] - 1, y, x, C->stream); });
    if (st) return st;
    st = run(C, 5, 1, [&] { return launch_solve_axis(C->solve[which][1], C->p[1] - 1, x, x, C->stream); });
    if (st) return st;
    return run(C, 6, 1, [&] { return launch_solve_axis(C->solve[which][2], C->p[2] - 1, x, x, C->stream); });
}

int dot_impl(smx_ctx* C, const double* x, const double* y, long long n, int slot) {
    return run(C, 7, 2, [&] { return launch_dot(x, y, n, C->partial, C->dots + slot, C->stream); });
}

// ---- reverse step helpers
// y += M x (the Hodge kernels scatter with atomics, so no zeroing means accumulation)
int hodge_apply_acc_impl(smx_ctx* C, int h, const double* x, double* y) {
    if (C->hodge[h].mode == 0) return run(C, 2, 1, [&] { return launch_hodge_block(C->hb[h], x, y, C->stream); });
    return run(C, 3, 1, [&] { return launch_hodge_quad(C->hq[h], x, y, C->stream); });
}

// x = K^{-T} y: the pairing sweeps with the transposed 1D factors
int solveT_impl(smx_ctx* C, int which, const double* y, double* x) {
    int st = run(C, 4, 1, [&] { return launch_solve_axis(C->solveT[which][0], C->p[0] - 1, y, x, C->stream); });
    if (st) return st;
    st = run(C, 5, 1, [&] { return launch_solve_axis(C->solveT[which][1], C->p[1] - 1, x, x, C->stream); });
    if (st) return st;
    return run(C, 6, 1, [&] { return launch_solve_axis(C->solveT[which][2], C->p[2] - 1, x, x, C->stream); });
}

// out[c] += z^T (dM~/deps_c) d for every permittivity block c
int pair_impl(smx_ctx* C, const double* z, const double* d, double* out) {
    if (C->hodge[1].mode == 0)
        return run(C, 19, 1, [&] { return launch_hodge_block_pair(C->hb[1], C->pair, z, d, out, C->stream); });
    return run(C, 19, 1, [&] { return launch_hodge_quad_pair(C->hq[1], C->pair, z, d, out, C->stream); });
}

// ---- mixed precision: FP32 operators on the FP64 state
// FP32 Hodge star from the FP64 2-form x into out (h = 0: h32 = K~_1^{-1} M^2 b;
// h = 1: e32 = K_1^{-1} M~^2 d), same algorithms as the FP64 path.  out64
// (optional) also receives the result widened to FP64: written by the last
// tensor-core sweep itself, else by a cast kernel.
// scratch = M x: FP32 element (or tile) contributions, summed in FP64 -- with up to
// (p+1)^3 contributions per coefficient an FP32 sum would lose accuracy where
// they cancel (block-Kronecker or quadrature Hodge, by the field's mode).
// Longest line of any field (entries along one axis).
int max_line_len(const smx_ctx* C) {
    int maxlen = 0;
    for (int a = 0; a < 3; ++a) maxlen = std::max(maxlen, kind_dim(P0, C->p[a], C->nel[a]) + 1);
    return maxlen;
}

// The mixed forms' dense line operators: the four-digit tensor-core kernel for SMX_MODE_TENSOR,
// and for SMX_MODE_AUTO once lines reach 32 entries; else the FP32 CUDA-core product.  Measured
// per step (tensor against CUDA cores): 0.122 against 0.139 ms at p = 3, 64^3; 0.579 against
// 0.555 ms at p = 3, 32^3, where only the tensor-core products keep the curved pulse within
// 1e-5 of FP64 over 500 steps (5.3e-6 against 1.3e-5); 0.060 against 0.032 ms at p = 2, 8^3.
bool mixed_tensor(const smx_ctx* C) {
    return C->mode_kernel == SMX_MODE_TENSOR || (C->mode_kernel == SMX_MODE_AUTO && max_line_len(C) >= 32);
}

int mass_f32(smx_ctx* C, int h, const double* x, bool prezeroed) {
    const long long ntot = C->fld[kFieldOfHodge[h]].total;
    if (!prezeroed) {
        const int st = run(C, 20, 1, [&] { return launch_zero(C->scratch, ntot, C->stream); });
        if (st) return st;
    }
    if (C->hodge[h].mode == 1)
        return run(C, 18, 1, [&] { return launch_hodge_quad_f32(C->hq32[h], x, C->scratch, C->stream); });
    return run(C, 13, 1, [&] { return launch_hodge_block_f32(C->hb32[h], x, nullptr, C->scratch, C->stream); });
}

// The mixed step fuses the mass of a separable star into its line operators (A^{-1} M);
// the refined step always applies the mass on its own.
bool fused_star(const smx_ctx* C, int h) { return C->hodge[h].separable && C->precision == SMX_MIXED; }

int hodge_star_f32_impl(smx_ctx* C, int h, const double* x, float* out, double* out64 = nullptr,
                        bool prezeroed = false) {
    int st;
    const long long ntot = C->fld[kFieldOfHodge[h]].total;
    auto widen = [&]() {
        return out64 ? run(C, 17, 1, [&] { return launch_cast_f2d(out, out64, ntot, C->stream); }) : SMX_OK;
    };
    if (C->use_mode) {
        // dense mode products: A^{-1} M per axis (separable) or block mass + A^{-1} per axis
        const double* x64 = x;
        const float* x32 = nullptr;
        if (!fused_star(C, h)) {
            if ((st = mass_f32(C, h, x, prezeroed))) return st;
            x64 = C->scratch;
        }
        // AUTO: the four-digit tensor-core kernel from 32-entry lines (mixed_tensor: more accurate
        // than the FP32 CUDA-core product, and faster there)
        const bool tc = mixed_tensor(C);
        auto pass = [&](int a, const double* i64, const float* i32, double* o64) {
            return run(C, (tc ? 24 : 14) + a, 1, [&] {
                return tc ? launch_mode_digit_f32(C->mdg[h][a], i64, i32, out, o64, C->stream)
                          : launch_mode_f32(C->md32[h][a], i64, i32, out, C->stream);
            });
        };
        if ((st = pass(0, x64, x32, nullptr))) return st;
        if ((st = pass(1, nullptr, out, nullptr))) return st;
        if ((st = pass(2, nullptr, out, tc ? out64 : nullptr))) return st;
        return tc ? SMX_OK : widen();
    }
    if (fused_star(C, h)) {
        st = run(C, 14, 1, [&] { return launch_line_f32(C->ln32[h][0], C->p[0] - 1, true, x, nullptr, out, C->stream); });
        if (st) return st;
        st = run(C, 15, 1, [&] { return launch_line_f32(C->ln32[h][1], C->p[1] - 1, true, nullptr, out, out, C->stream); });
        if (st) return st;
        st = run(C, 16, 1, [&] { return launch_line_f32(C->ln32[h][2], C->p[2] - 1, true, nullptr, out, out, C->stream); });
        return st ? st : widen();
    }
    if ((st = mass_f32(C, h, x, prezeroed))) return st;
    st = run(C, 14, 1, [&] { return launch_line_f32(C->ln32[h][0], C->p[0] - 1, false, C->scratch, nullptr, out, C->stream); });
    if (st) return st;
    st = run(C, 15, 1, [&] { return launch_line_f32(C->ln32[h][1], C->p[1] - 1, false, nullptr, out, out, C->stream); });
    if (st) return st;
    st = run(C, 16, 1, [&] { return launch_line_f32(C->ln32[h][2], C->p[2] - 1, false, nullptr, out, out, C->stream); });
    return st ? st : widen();
}

int step_mixed(smx_ctx* C, double* d, double* b, double* e, double* h, const double* jhat, const double* amp, double dt,
               int nsteps) {
    const DevField &FE = C->fld[SMX_FIELD_E], &FB = C->fld[SMX_FIELD_B], &FH = C->fld[SMX_FIELD_H],
                   &FD = C->fld[SMX_FIELD_D];
    int st = run(C, 17, 1, [&] { return launch_cast_d2f(e, C->e32, C->N_e, C->stream); });
    if (st) return st;
    // the curl before a star that accumulates a mass apply also clears that accumulator
    const bool zH = !fused_star(C, 0), zD = !fused_star(C, 1);
    double* zeroH = zH ? C->scratch : nullptr;
    double* zeroD = zD ? C->scratch : nullptr;
    st = run(C, 11, 1, [&] {
        return launch_curl_f32(false, FE, FB, C->e32, b, -0.5 * dt, nullptr, nullptr, 0, 0.0, C->stream, zeroH);
    });
    if (st) return st;
    for (int n = 0; n < nsteps; ++n) {
        const bool last = n + 1 == nsteps;  // the last stars also write the FP64 1-forms h and e
        if ((st = hodge_star_f32_impl(C, 0, b, C->h32, last ? h : nullptr, zH))) return st;
        st = run(C, 12, 1, [&] {
            return launch_curl_f32(true, FH, FD, C->h32, d, dt, jhat, amp, n, 0.0, C->stream, zeroD);
        });
        if (st) return st;
        if ((st = hodge_star_f32_impl(C, 1, d, C->e32, last ? e : nullptr, zD))) return st;
        const double alpha = (n + 1 == nsteps) ? -0.5 * dt : -dt;
        st = run(C, 11, 1, [&] {
            return launch_curl_f32(false, FE, FB, C->e32, b, alpha, nullptr, nullptr, 0, 0.0, C->stream, zeroH);
        });
        if (st) return st;
    }
    return SMX_OK;
}

// out (FP32) = K^{-1} y by the mixed step's line operators (dense A^{-1} products on the
// FP32 CUDA cores or the four-digit tensor-core kernel, or FP32 banded recurrences for
// lines longer than 80); y is FP64.
int solve_f32_impl(smx_ctx* C, int h, const double* y, float* out) {
    int st;
    if (C->use_mode) {
        const bool tc = mixed_tensor(C);
        for (int a = 0; a < 3; ++a) {
            st = run(C, (tc ? 24 : 14) + a, 1, [&] {
                const double* i64 = a == 0 ? y : nullptr;
                const float* i32 = a == 0 ? nullptr : out;
                return tc ? launch_mode_digit_f32(C->mdg[h][a], i64, i32, out, nullptr, C->stream)
                          : launch_mode_f32(C->md32[h][a], i64, i32, out, C->stream);
            });
            if (st) return st;
        }
        return SMX_OK;
    }
    for (int a = 0; a < 3; ++a) {
        st = run(C, 14 + a, 1, [&] {
            return launch_line_f32(C->ln32[h][a], C->p[a] - 1, false, a == 0 ? y : nullptr, a == 0 ? nullptr : out,
                                   out, C->stream);
        });
        if (st) return st;
    }
    return SMX_OK;
}

// The refined mixed Hodge star (SMX_MIXED_REFINED): y = M x (FP32 element
// contributions summed in FP64), x0 = K^{-1} y in FP32, the residual
// r = y - K x0 formed in FP64 (three banded passes of the 1D pairing factors on
// the FP64 pipe), one correction c = K^{-1} r in FP32, out = x0 + c in FP64.
int star_refined(smx_ctx* C, int h, const double* x, double* out, bool prezeroed) {
    int st;
    const long long ntot = C->fld[kFieldOfHodge[h]].total;
    float* x0 = h == 0 ? C->h32 : C->e32;
    if ((st = mass_f32(C, h, x, prezeroed))) return st;  // y in scratch
    if ((st = solve_f32_impl(C, h, C->scratch, x0))) return st;
    // r = y - (A_z (x) A_y (x) A_x) x0: t64 = A_x x0, scratch2 = A_y t64, t64 = y - A_z scratch2
    if ((st = run(C, 27, 1, [&] { return launch_band_apply(C->band[h][0], nullptr, x0, nullptr, C->t64, C->stream); })))
        return st;
    if ((st = run(C, 27, 1, [&] { return launch_band_apply(C->band[h][1], C->t64, nullptr, nullptr, C->scratch2, C->stream); })))
        return st;
    if ((st = run(C, 27, 1, [&] {
             return launch_band_apply(C->band[h][2], C->scratch2, nullptr, C->scratch, C->t64, C->stream);
         })))
        return st;
    if ((st = solve_f32_impl(C, h, C->t64, C->y32))) return st;
    return run(C, 17, 1, [&] { return launch_refine_sum(x0, C->y32, out, ntot, C->stream); });
}

// Refined mixed steps: FP64 state and curls (d, b, e, h all FP64), refined stars.
int step_refined(smx_ctx* C, double* d, double* b, double* e, double* h, const double* jhat, const double* amp,
                 double dt, int nsteps);

int hodge_star_impl(smx_ctx* C, int h, const double* x, double* out, bool prezeroed = false);

// nsteps kick-drift-kick steps enqueued kernel by kernel (the inner half kicks of b merged).
int step_eager(smx_ctx* C, double* d, double* b, double* e, double* h, const double* jhat, const double* amp, double dt,
               int nsteps) {
    if (C->precision == SMX_MIXED) return step_mixed(C, d, b, e, h, jhat, amp, dt, nsteps);
    if (C->precision == SMX_MIXED_REFINED) return step_refined(C, d, b, e, h, jhat, amp, dt, nsteps);
    // the curl before a star that accumulates a mass apply also clears that accumulator
    const bool zH = !C->hodge[0].separable, zD = !C->hodge[1].separable;
    double* zeroH = zH ? C->scratch : nullptr;
    double* zeroD = zD ? C->scratch : nullptr;
    int st = curl_primal_impl(C, e, b, -0.5 * dt, zeroH);
    if (st) return st;
    for (int n = 0; n < nsteps; ++n) {
        if ((st = hodge_star_impl(C, 0, b, h, zH))) return st;  // h = K~_1^{-1} M^2_{1/mu} b
        if ((st = curl_dual_impl(C, h, d, dt, jhat, amp, n, 0.0, zeroD))) return st;
        if ((st = hodge_star_impl(C, 1, d, e, zD))) return st;  // e = K_1^{-1} M~^2_{1/eps} d
        if ((st = curl_primal_impl(C, e, b, (n + 1 == nsteps) ? -0.5 * dt : -dt, zeroH))) return st;
    }
    return SMX_OK;
}

int step_refined(smx_ctx* C, double* d, double* b, double* e, double* h, const double* jhat, const double* amp,
                 double dt, int nsteps) {
    double* zero = C->scratch;  // every refined star starts with a mass apply into the scratch vector
    int st = curl_primal_impl(C, e, b, -0.5 * dt, zero);
    if (st) return st;
    for (int n = 0; n < nsteps; ++n) {
        if ((st = star_refined(C, 0, b, h, true))) return st;
        if ((st = curl_dual_impl(C, h, d, dt, jhat, amp, n, 0.0, zero))) return st;
        if ((st = star_refined(C, 1, d, e, true))) return st;
        if ((st = curl_primal_impl(C, e, b, (n + 1 == nsteps) ? -0.5 * dt : -dt, zero))) return st;
    }
    return SMX_OK;
}

// ---- refined mixed reverse step: the transposed stars S^T = M K^{-T} in the arithmetic of the
// refined forward step.  x = K^{-T} y (which = 0: K_1^T, 1: K~_1^T; y, x FP64, distinct): x0 by
// FP32 banded sweeps with the transposed factors, r = y - K^T x0 by FP64 banded passes, one FP32
// correction, x = x0 + c.  Uses e32 / h32, y32, t64 and the state vectors as scratch.
int solveT_refined(smx_ctx* C, int which, const double* y, double* x) {
    const int h = which == 0 ? 1 : 0;
    const long long n = C->fld[which == 0 ? SMX_FIELD_D : SMX_FIELD_B].total;
    float* x0 = which == 0 ? C->e32 : C->h32;
    double* t2 = C->state;
    int st;
    auto sweeps = [&](const double* in64, float* out) {
        for (int a = 0; a < 3; ++a) {
            const int r = run(C, 14 + a, 1, [&] {
                return launch_line_f32(C->ln32T[which][a], C->p[a] - 1, false, a == 0 ? in64 : nullptr,
                                       a == 0 ? nullptr : out, out, C->stream);
            });
            if (r) return r;
        }
        return SMX_OK;
    };
    (void)h;
    if ((st = sweeps(y, x0))) return st;
    if ((st = run(C, 27, 1, [&] { return launch_band_apply(C->bandT[which][0], nullptr, x0, nullptr, C->t64, C->stream); })))
        return st;
    if ((st = run(C, 27, 1, [&] { return launch_band_apply(C->bandT[which][1], C->t64, nullptr, nullptr, t2, C->stream); })))
        return st;
    if ((st = run(C, 27, 1, [&] { return launch_band_apply(C->bandT[which][2], t2, nullptr, y, C->t64, C->stream); })))
        return st;
    if ((st = sweeps(C->t64, C->y32))) return st;
    return run(C, 17, 1, [&] { return launch_refine_sum(x0, C->y32, x, n, C->stream); });
}

// out += M x (h = 0: M^2_{1/mu}, 1: M~^2_{1/eps}) with the mixed step's FP32 mass kernels (element
// contributions summed in FP64) for a refined context, else the FP64 mass kernels.
int mass_acc_any(smx_ctx* C, int h, const double* x, double* out) {
    if (C->precision != SMX_MIXED_REFINED) return hodge_apply_acc_impl(C, h, x, out);
    int st = mass_f32(C, h, x, false);  // into the scratch vector
    if (st) return st;
    const long long n = C->fld[kFieldOfHodge[h]].total;
    return run(C, 20, 1, [&] { return launch_axpy(C->scratch, out, 1.0, n, C->stream); });
}

int solveT_any(smx_ctx* C, int which, const double* y, double* x) {
    return C->precision == SMX_MIXED_REFINED ? solveT_refined(C, which, y, x) : solveT_impl(C, which, y, x);
}

// ---- scheme 1 (Sec. 3.3): Hodge stars by mass-matrix solves, for comparison with scheme 2
// y = K^T x along the three axes: k = 0 K_2 = K~_1^T (x in the B layout, y in H), k = 1
// K~_2 = K_1^T (x in D, y in E); t1, t2 are scratch vectors (all four distinct).
int s1_pair_t(smx_ctx* C, int k, const double* x, double* y, double* t1, double* t2) {
    int st = run(C, 27, 1, [&] { return launch_band_apply(C->kt[k][0], x, nullptr, nullptr, t1, C->stream); });
    if (st) return st;
    st = run(C, 27, 1, [&] { return launch_band_apply(C->kt[k][1], t1, nullptr, nullptr, t2, C->stream); });
    if (st) return st;
    return run(C, 27, 1, [&] { return launch_band_apply(C->kt[k][2], t2, nullptr, nullptr, y, C->stream); });
}

// y = M x for the 1-form mass k (0: M~^1_mu, 1: M^1_eps), y overwritten
int s1_mass(smx_ctx* C, int k, const double* x, double* y) {
    const long long n = C->fld[k == 0 ? SMX_FIELD_H : SMX_FIELD_E].total;
    int st = run(C, 20, 1, [&] { return launch_zero(y, n, C->stream); });
    if (st) return st;
    if (C->hodge1[k].mode == 0) return run(C, 2, 1, [&] { return launch_hodge_block(C->hb1[k], x, y, C->stream); });
    return run(C, 3, 1, [&] { return launch_hodge_quad(C->hq1[k], x, y, C->stream); });
}

// x = P^{-1} y: the unit-material Kronecker mass solved by three banded sweeps (in place when x == y)
int s1_precond(smx_ctx* C, int k, const double* y, double* x) {
    int st = run(C, 4, 1, [&] { return launch_solve_axis(C->pre1[k][0], C->p[0], y, x, C->stream); });
    if (st) return st;
    st = run(C, 5, 1, [&] { return launch_solve_axis(C->pre1[k][1], C->p[1], x, x, C->stream); });
    if (st) return st;
    return run(C, 6, 1, [&] { return launch_solve_axis(C->pre1[k][2], C->p[2], x, x, C->stream); });
}

// x = M^{-1} y by conjugate gradients preconditioned with the unit-material Kronecker mass
// (for constant material on the identity map the mass is that preconditioner times the
// constant: one iteration), to ||y - M x|| <= tol ||y||.  The residual is read back after the
// first iteration and then every 4 (the only host synchronisations); *iters receives the
// iterations used.  y must not be a PCG vector.
int s1_pcg(smx_ctx* C, int k, const double* y, double* x, double tol, int maxit, int* iters) {
    const long long n = C->fld[k == 0 ? SMX_FIELD_H : SMX_FIELD_E].total;
    double *r = C->s1v[0], *z = C->s1v[1], *pv = C->s1v[2], *Ap = C->scratch2, *cg = C->cg;
    int st;
    auto dot = [&](const double* a, const double* b, int slot) {
        return run(C, 7, 2, [&] { return launch_dot(a, b, n, C->partial, cg + slot, C->stream); });
    };
    auto converged = [&](bool& done) {
        double h[kCgCount];
        CK(cudaMemcpyAsync(h, cg, sizeof h, cudaMemcpyDeviceToHost, C->stream));
        CK(cudaStreamSynchronize(C->stream));
        if (!std::isfinite(h[kCgRr]) || !std::isfinite(h[kCgYy])) return SMX_ENONFINITE;
        done = h[kCgRr] <= tol * tol * h[kCgYy];
        return SMX_OK;
    };
    if ((st = s1_precond(C, k, y, x))) return st;
    if ((st = s1_mass(C, k, x, r))) return st;
    if ((st = run(C, 20, 1, [&] { return launch_sub_from(y, r, n, C->stream); }))) return st;
    if ((st = dot(y, y, kCgYy)) || (st = dot(r, r, kCgRr))) return st;
    bool done = false;
    if ((st = converged(done))) return st;
    int it = 0;
    if (!done) {
        if ((st = s1_precond(C, k, r, z))) return st;
        if ((st = dot(r, z, kCgRz))) return st;
        if ((st = run(C, 20, 1, [&] { return launch_copy(z, pv, n, C->stream); }))) return st;
        while (it < maxit) {
            ++it;
            if ((st = s1_mass(C, k, pv, Ap))) return st;
            if ((st = dot(pv, Ap, kCgPAp))) return st;
            if ((st = run(C, 20, 1, [&] { return launch_cg_xr(x, r, pv, Ap, cg, n, C->stream); }))) return st;
            if (it == 1 || it % 4 == 0 || it == maxit) {
                if ((st = dot(r, r, kCgRr))) return st;
                if ((st = converged(done))) return st;
                if (done) break;
            }
            if ((st = s1_precond(C, k, r, z))) return st;
            if ((st = dot(r, z, kCgRzNew))) return st;
            if ((st = run(C, 20, 2, [&] { return launch_cg_p(pv, z, cg, n, C->stream); }))) return st;
        }
    }
    if (iters) *iters = it;
    return done ? SMX_OK : SMX_ESINGULAR;
}

// One Hodge star of scheme 1: h = (M~^1_mu)^{-1} K_2 b (k = 0) or e = (M^1_eps)^{-1} K~_2 d (k = 1)
int s1_star(smx_ctx* C, int k, const double* x, double* out, double tol, int maxit, int* iters) {
    int st = s1_pair_t(C, k, x, C->scratch, C->s1v[0], C->s1v[1]);
    if (st) return st;
    return s1_pcg(C, k, C->scratch, out, tol, maxit, iters);
}

// One discrete Hodge star of scheme 2 (Eq. discrete2_hodge_mu for h = 0,
// Eq. discrete2_hodge_eps for h = 1): three fused mass+solve line passes when
// the field's mass is a single Kronecker product, else mass apply into the
// scratch vector followed by the three pairing sweeps.
int hodge_star_impl(smx_ctx* C, int h, const double* x, double* out, bool prezeroed) {
    const int which = h == 0 ? 1 : 0;
    // SMX_MODE_AUTO takes, per star, the kernel measured faster on GB300.  The
    // banded recurrences cost about n (2(2d+1) + 4 KL + 1) dependent FP64 steps
    // per line (fused mass + solve) or n (4 KL + 1) (pairing sweep); the digit
    // kernel costs about 12 us of fixed latency plus time proportional to the
    // lines.  Measured: the digit passes win for a separable star once lines
    // reach about 48 entries, and for the pairing sweeps too from p = 4 (KL = 3)
    // or from 64 entries (p = 3, 64^3: 19-21 us against 22-25 us per pass).
    const int maxlen = max_line_len(C);
    int maxkl = 0;
    for (int a = 0; a < 3; ++a) maxkl = std::max(maxkl, C->p[a] - 1);
    const bool auto_digit = maxlen >= 48 && (C->hodge[h].separable || maxkl >= 3 || maxlen >= 64);
    const bool digit = C->use_digit && C->precision == SMX_FP64 &&
                       (C->mode_kernel == SMX_MODE_TENSOR || (C->mode_kernel == SMX_MODE_AUTO && auto_digit));
    if (digit) {
        // dense line operators on the tensor cores: A^{-1} M per axis (separable), or
        // the mass apply followed by A^{-1} per axis
        const double* src = x;
        if (!C->hodge[h].separable) {
            const int st = hodge_apply_impl(C, h, x, C->scratch, prezeroed);
            if (st) return st;
            src = C->scratch;
        }
        for (int a = 0; a < 3; ++a) {
            const int st =
                run(C, 21 + a, 1, [&] { return launch_mode_digit(C->mdg[h][a], a == 0 ? src : out, out, C->stream); });
            if (st) return st;
        }
        return SMX_OK;
    }
    if (C->hodge[h].separable) {
        int st = run(C, 8, 1, [&] { return launch_mass_solve_axis(C->ms[h][0], C->p[0] - 1, x, out, C->stream); });
        if (st) return st;
        st = run(C, 9, 1, [&] { return launch_mass_solve_axis(C->ms[h][1], C->p[1] - 1, out, out, C->stream); });
        if (st) return st;
        return run(C, 10, 1, [&] { return launch_mass_solve_axis(C->ms[h][2], C->p[2] - 1, out, out, C->stream); });
    }
    const int st = hodge_apply_impl(C, h, x, C->scratch, prezeroed);
    if (st) return st;
    return solve_impl(C, which, C->scratch, out);
}

}  // namespace

extern "C" {

const char* smx_strerror(int s) {
    switch (s) {
        case SMX_OK: return "ok";
        case SMX_EINVAL: return "invalid argument";
        case SMX_EGEOM: return "geometry map not orientation preserving (det J <= 0)";
        case SMX_EMAT: return "material not finite and positive";
        case SMX_ECUDA: return "CUDA runtime error";
        case SMX_ENONFINITE: return "non-finite value in the fields";
        case SMX_ESTATE: return "workspace missing or too small";
        case SMX_ENOMEM: return "host allocation failed";
        case SMX_ESINGULAR: return "singular 1D pairing factor";
        case SMX_ENOSPACE: return "problem larger than the fixed no-alloc device array";
        case SMX_ETIMEOUT: return "a device-side wait gave up after its time limit";
        default: return "unknown status";
    }
}

int smx_create(const smx_params* P, smx_ctx** out) {
    if (!P || !out) return SMX_EINVAL;
    *out = nullptr;
    for (int a = 0; a < 3; ++a) {
        if (P->p[a] < 2 || P->p[a] > kPMax) return SMX_EINVAL;
        if (P->nel[a] < 1 || P->nel[a] > 800) return SMX_EINVAL;
    }
    if (P->geometry != SMX_GEOM_IDENTITY && P->geometry != SMX_GEOM_SINE_BUMP && P->geometry != SMX_GEOM_CALLBACK)
        return SMX_EINVAL;
    if (P->geometry == SMX_GEOM_CALLBACK && !P->geom_fn) return SMX_EINVAL;
    if (!std::isfinite(P->geom_amplitude)) return SMX_EINVAL;
    int st = check_material(P->eps, P->nel);
    if (st) return st;
    st = check_material(P->mu, P->nel);
    if (st) return st;
    smx_ctx* C = new (std::nothrow) smx_ctx();
    if (!C) return SMX_ENOMEM;
    C->uid = g_next_uid.fetch_add(1);
    try {
        for (int a = 0; a < 3; ++a) {
            C->p[a] = P->p[a];
            C->nel[a] = P->nel[a];
        }
        C->geometry = P->geometry;
        C->amp = P->geom_amplitude;
        C->gmap.kind = P->geometry;
        C->gmap.amp = P->geom_amplitude;
        C->gmap.fn = P->geometry == SMX_GEOM_CALLBACK ? P->geom_fn : nullptr;
        C->gmap.user = P->geom_user;
        if (P->eps.kind == SMX_MAT_BLOCKS) {
            C->eps_blocks = true;
            for (int a = 0; a < 3; ++a) {
                C->eps_nb[a] = P->eps.blocks[a];
                C->eps_epb[a] = P->nel[a] / P->eps.blocks[a];
            }
            C->eps_vals.assign(P->eps.block_values,
                               P->eps.block_values + (size_t)C->eps_nb[0] * C->eps_nb[1] * C->eps_nb[2]);
        }
        for (int f = 0; f < 4; ++f) {
            long long off = 0;
            for (int c = 0; c < 3; ++c) {
                for (int a = 0; a < 3; ++a) C->fld[f].c[c].n[a] = kind_dim(kFieldKinds[f][c][a], C->p[a], C->nel[a]);
                C->fld[f].c[c].off = off;
                off += (long long)C->fld[f].c[c].n[0] * C->fld[f].c[c].n[1] * C->fld[f].c[c].n[2];
            }
            C->fld[f].total = off;
        }
        C->N_e = C->fld[SMX_FIELD_E].total;
        C->N_h = C->fld[SMX_FIELD_H].total;
        // 1D factors (Sec. 4.1) and their banded LU (Sec. 4.3, Table 1 setup)
        for (int a = 0; a < 3; ++a) {
            const int p = C->p[a], nel = C->nel[a];
            const std::vector<double> G = pairing_matrix(D1, P0, p, nel);
            const std::vector<double> M = pairing_matrix(D0, P1, p, nel);
            const int nG = kind_dim(D1, p, nel), nM = kind_dim(D0, p, nel);
            if (!is_banded(G, nG, p - 1) || !is_banded(M, nM, p - 1)) {
                delete C;
                return SMX_ESINGULAR;
            }
            const std::vector<double>* mats[4] = {&G, &M, nullptr, nullptr};
            const std::vector<double> Gt = transpose(G, nG), Mt = transpose(M, nM);
            mats[2] = &Gt;
            mats[3] = &Mt;
            const int ns[4] = {nG, nM, nG, nM};
            for (int w = 0; w < 4; ++w) {
                if (!band_lu(*mats[w], ns[w], p - 1, p - 1, C->fac[a][w])) {
                    delete C;
                    return SMX_ESINGULAR;
                }
                // band rows A(m, m - kl .. m + kl) of the factor itself (the refined step's residual)
                const int n = ns[w], kl = p - 1, W = 2 * kl + 1;
                std::vector<double>& R = C->band_rows[a][w];
                R.assign((size_t)n * W, 0.0);
                for (int m = 0; m < n; ++m)
                    for (int q = 0; q < W; ++q) {
                        const int j = m - kl + q;
                        if (j >= 0 && j < n) R[(size_t)m * W + q] = (*mats[w])[(size_t)m * n + j];
                    }
            }
        }
        // Hodge tables: block Kronecker on the identity map with constant or block material
        const smx_material* mats[2] = {&P->mu, &P->eps};
        for (int h = 0; h < 2; ++h) {
            const bool block = C->geometry == SMX_GEOM_IDENTITY && mats[h]->kind != SMX_MAT_POINTWISE;
            C->hodge[h].mode = block ? 0 : 1;
            st = block ? build_hodge_block(C, h, *mats[h]) : build_hodge_quad(C, h, *mats[h]);
            if (st) {
                delete C;
                return st;
            }
            if (block && mats[h]->kind == SMX_MAT_CONST) build_separable(C, h, 1.0 / mats[h]->value);
        }
        if (P->scheme1) {
            // scheme 1: 1-form masses weighted by the material itself (Eq. discrete1_hodge_mu / _eps),
            // block-Kronecker on the identity map, quadrature with the 1-form metric otherwise
            for (int a = 0; a < 3; ++a)
                if (C->p[a] > 5) {
                    delete C;
                    return SMX_EINVAL;
                }
            C->s1 = true;
            const smx_material* mats1[2] = {&P->mu, &P->eps};
            const int flds1[2] = {SMX_FIELD_H, SMX_FIELD_E};
            for (int k = 0; k < 2; ++k) {
                const bool block = C->geometry == SMX_GEOM_IDENTITY && mats1[k]->kind != SMX_MAT_POINTWISE;
                C->hodge1[k].mode = block ? 0 : 1;
                st = block ? build_hodge_block_t(C, C->hodge1[k], flds1[k], *mats1[k], false)
                           : build_hodge_quad_t(C, C->hodge1[k], *mats1[k], true);
                if (st) {
                    delete C;
                    return st;
                }
            }
            // the preconditioner: unit-material Kronecker 1D masses of every kind, banded LU with
            // half-bandwidth p on both sides (the widest kind; narrower kinds carry zeros)
            for (int a = 0; a < 3; ++a)
                for (int kind = 0; kind < 4; ++kind) {
                    const int pa = C->p[a], nel = C->nel[a], d = kind_degree(kind, pa), off = kind_offset(kind);
                    const int dim = kind_dim(kind, pa, nel);
                    std::vector<double> M((size_t)dim * dim, 0.0);
                    for (int e = 0; e < nel; ++e) {
                        const std::vector<double> Me = element_mass(kind, pa, nel, e);
                        for (int r = 0; r <= d; ++r)
                            for (int q = 0; q <= d; ++q) {
                                const int i = e + r + off, j = e + q + off;
                                if (i >= 0 && i < dim && j >= 0 && j < dim) M[(size_t)i * dim + j] += Me[r * (d + 1) + q];
                            }
                    }
                    if (!band_lu(M, dim, pa, pa, C->mfac[a][kind])) {
                        delete C;
                        return SMX_ESINGULAR;
                    }
                }
        }
        if (P->precision != SMX_FP64 && P->precision != SMX_MIXED && P->precision != SMX_MIXED_REFINED) {
            delete C;
            return SMX_EINVAL;
        }
        C->precision = P->precision;
        // pack the tables
        for (int a = 0; a < 3; ++a)
            for (int w = 0; w < 4; ++w) {
                C->o_fac[a][w][0] = C->blob.add(C->fac[a][w].L);
                C->o_fac[a][w][1] = C->blob.add(C->fac[a][w].U);
                C->o_fac[a][w][2] = C->blob.add(C->fac[a][w].dinv);
            }
        for (int h = 0; h < 2; ++h) {
            HodgeHost& H = C->hodge[h];
            if (H.mode == 0) {
                for (int a = 0; a < 3; ++a) {
                    H.o_tf0[a] = C->blob.add(H.tf0[a]);
                    H.o_tlen[a] = C->blob.add(H.tlen[a]);
                    H.o_tmat[a] = C->blob.add(H.tmat[a]);
                }
                H.o_gamma = C->blob.add(H.gamma);
                if (H.separable)
                    for (int a = 0; a < 3; ++a)
                        for (int kind = 0; kind < 4; ++kind) H.o_lmass[a][kind] = C->blob.add(H.lmass[a][kind]);
            } else {
                for (int a = 0; a < 3; ++a) H.o_bval[a] = C->blob.add(H.bval[a]);
                H.o_G = C->blob.add(H.G);
                if (C->precision != SMX_FP64) {  // the mixed step's FP32 (hi, lo) copies
                    for (int a = 0; a < 3; ++a) C->o_bval32[h][a] = C->blob.add(split_pairs(H.bval[a]));
                    C->o_G32[h] = C->blob.add(split_pairs(H.G));
                }
                H.G.clear();
                H.G.shrink_to_fit();
            }
        }
        if (C->precision == SMX_MIXED_REFINED || C->s1)
            for (int a = 0; a < 3; ++a)
                for (int w = 0; w < 4; ++w) C->o_band[a][w] = C->blob.add(C->band_rows[a][w]);
        if (C->s1) {
            for (int k = 0; k < 2; ++k) {
                HodgeHost& H = C->hodge1[k];
                if (H.mode == 0) {
                    for (int a = 0; a < 3; ++a) {
                        H.o_tf0[a] = C->blob.add(H.tf0[a]);
                        H.o_tlen[a] = C->blob.add(H.tlen[a]);
                        H.o_tmat[a] = C->blob.add(H.tmat[a]);
                    }
                    H.o_gamma = C->blob.add(H.gamma);
                } else {
                    for (int a = 0; a < 3; ++a) H.o_bval[a] = C->blob.add(H.bval[a]);
                    H.o_G = C->blob.add(H.G);
                    H.G.clear();
                    H.G.shrink_to_fit();
                }
            }
            for (int a = 0; a < 3; ++a)
                for (int kind = 0; kind < 4; ++kind) {
                    C->o_mfac[a][kind][0] = C->blob.add(C->mfac[a][kind].L);
                    C->o_mfac[a][kind][1] = C->blob.add(C->mfac[a][kind].U);
                    C->o_mfac[a][kind][2] = C->blob.add(C->mfac[a][kind].dinv);
                }
        }
        if (C->precision != SMX_FP64) {
            // FP32 (hi, lo) copies of every operator table of the mixed step
            for (int a = 0; a < 3; ++a)
                for (int w = 0; w < 4; ++w) {
                    C->o_fac32[a][w][0] = C->blob.add(split_pairs(C->fac[a][w].L));
                    C->o_fac32[a][w][1] = C->blob.add(split_pairs(C->fac[a][w].U));
                    C->o_fac32[a][w][2] = C->blob.add(split_pairs(C->fac[a][w].dinv));
                }
            for (int h = 0; h < 2; ++h) {
                HodgeHost& H = C->hodge[h];
                for (int a = 0; a < 3; ++a) C->o_tmat32[h][a] = C->blob.add(split_pairs(H.tmat[a]));
                if (H.separable)
                    for (int a = 0; a < 3; ++a)
                        for (int kind = 0; kind < 4; ++kind)
                            C->o_lmass32[h][a][kind] = C->blob.add(split_pairs(H.lmass[a][kind]));
            }
        }
        // dense line operators for the mode-product sweeps: A^{-1}, or A^{-1} M (separable
        // star) -- as FP32 pairs and BF16 parts (mixed step) or as digit planes (FP64 step)
        bool dense = true;
        for (int a = 0; a < 3; ++a)
            if (kind_dim(P0, C->p[a], C->nel[a]) + 1 > kModeMaxN) dense = false;
        if (dense) {
            C->use_mode = C->precision != SMX_FP64;
            C->use_digit = true;  // digit planes: 7 digits (FP64 step) or 4 (mixed step)
            const int nd = C->precision == SMX_FP64 ? kDigits : kDigitsF32;
            std::vector<double> inv[3][4];
            for (int a = 0; a < 3; ++a)
                for (int w = 0; w < 4; ++w) inv[a][w] = dense_inverse(C->fac[a][w]);
            for (int h = 0; h < 2; ++h) {
                const HodgeHost& H = C->hodge[h];
                const int fld = kFieldOfHodge[h], which = h == 0 ? 1 : 0;
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < 3; ++c) {
                        const int w = factor_index(which, c, a), kind = kFieldKinds[fld][c][a];
                        const int n = C->fac[a][w].n;
                        // a separable star of the FP64 and mixed steps fuses the mass: A^{-1} M; the
                        // refined step applies the mass on its own and needs A^{-1} for the residual
                        const std::vector<double> B =
                            (H.separable && C->precision != SMX_MIXED_REFINED)
                                ? dense_times_band(inv[a][w], H.lmass[a][kind], n, kind_degree(kind, C->p[a]))
                                : inv[a][w];
                        {
                            std::vector<uint16_t> planes;
                            std::vector<int32_t> rowexp;
                            digit_split_operator(B, n, mode_digit_npad(n), nd, planes, rowexp);
                            C->o_dig[h][a][c] = C->blob.add(planes);
                            C->o_dige[h][a][c] = C->blob.add(rowexp);
                        }
                        if (!C->use_mode) continue;
                        // CUDA-core kernel: transposed and zero padded to the kernel's output count,
                        // Bt[k][i] = B[i][k] for i < npad, so the staging is one contiguous copy
                        int maxn = 0;
                        for (int c2 = 0; c2 < 3; ++c2) maxn = std::max(maxn, C->fld[fld].c[c2].n[a]);
                        const int npad = mode_f32_npad(maxn);
                        std::vector<double> Bt((size_t)n * npad, 0.0);
                        for (int i = 0; i < n; ++i)
                            for (int k = 0; k < n; ++k) Bt[(size_t)k * npad + i] = B[(size_t)i * n + k];
                        C->o_mode32[h][a][c] = C->blob.add(split_pairs(Bt));
                    }
            }
        }
        if (C->eps_blocks) {  // per-block scale of the mass derivative (-1/eps) and the tiles' blocks
            std::vector<double> sc(C->eps_vals.size());
            for (size_t k = 0; k < sc.size(); ++k) sc[k] = -1.0 / C->eps_vals[k];
            C->o_pair_scale = C->blob.add(sc);
            C->o_tile_block = C->blob.add(C->hodge[1].tile_block);
        }
        layout(C);
    } catch (const std::bad_alloc&) {
        delete C;
        return SMX_ENOMEM;
    }
    *out = C;
    return SMX_OK;
}

int smx_destroy(smx_ctx* C) {
    if (C) {
        for (auto& t : C->timed) {
            cudaEventDestroy(t.a);
            cudaEventDestroy(t.b);
        }
        if (C->graph.exec) cudaGraphExecDestroy(C->graph.exec);
    }
    delete C;
    return SMX_OK;
}

int smx_sizes(const smx_ctx* C, int64_t* n_e, int64_t* n_h) {
    if (!C || !n_e || !n_h) return SMX_EINVAL;
    *n_e = C->N_e;
    *n_h = C->N_h;
    return SMX_OK;
}

int smx_comp_shape(const smx_ctx* C, int field, int comp, int64_t shape[3]) {
    if (!C || !shape || field < 0 || field > 3 || comp < 0 || comp > 2) return SMX_EINVAL;
    for (int a = 0; a < 3; ++a) shape[a] = C->fld[field].c[comp].n[a];
    return SMX_OK;
}

int smx_workspace_bytes(const smx_ctx* C, size_t* bytes) {
    if (!C || !bytes) return SMX_EINVAL;
    *bytes = C->total_bytes;
    return SMX_OK;
}

int smx_set_stream(smx_ctx* C, void* stream) {
    if (!C) return SMX_EINVAL;
    C->stream = static_cast<cudaStream_t>(stream);
    return SMX_OK;
}

int smx_bind_workspace(smx_ctx* C, void* dev, size_t bytes) {
    if (!C || !dev) return SMX_EINVAL;
    if (bytes < C->total_bytes || (reinterpret_cast<uintptr_t>(dev) & 255)) return SMX_ESTATE;
    unsigned char* ws = static_cast<unsigned char*>(dev);
    CK(cudaMemcpyAsync(ws, C->blob.bytes.data(), C->blob.bytes.size(), cudaMemcpyHostToDevice, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    C->ws = ws;
    if (C->graph.exec) {  // a captured step refers to the previous workspace
        cudaGraphExecDestroy(C->graph.exec);
        C->graph.exec = nullptr;
    }
    C->scratch = reinterpret_cast<double*>(ws + C->o_scratch);
    C->scratch2 = reinterpret_cast<double*>(ws + C->o_scratch2);
    C->partial = reinterpret_cast<double*>(ws + C->o_partial);
    C->dots = reinterpret_cast<double*>(ws + C->o_dots);
    C->status = reinterpret_cast<unsigned*>(ws + C->o_status);
    CK(cudaMemsetAsync(C->status, 0, sizeof(unsigned), C->stream));
    C->state = reinterpret_cast<double*>(ws + C->o_state);
    // transposed pairing sweeps (reverse step): K_1^T uses G^T, M^T in the D layout, K~_1^T uses G, M
    for (int which = 0; which < 2; ++which) {
        const int fld = which == 0 ? SMX_FIELD_D : SMX_FIELD_B;
        for (int a = 0; a < 3; ++a) {
            SolveArgs& S = C->solveT[which][a];
            S.field = C->fld[fld];
            S.axis = a;
            for (int c = 0; c < 3; ++c) {
                const int w = factor_index(which, c, a) ^ 2;  // 0 <-> 2 (G, G^T), 1 <-> 3 (M, M^T)
                S.f[c].L = reinterpret_cast<const double*>(ws + C->o_fac[a][w][0]);
                S.f[c].U = reinterpret_cast<const double*>(ws + C->o_fac[a][w][1]);
                S.f[c].dinv = reinterpret_cast<const double*>(ws + C->o_fac[a][w][2]);
                S.f[c].n = C->fac[a][w].n;
            }
        }
    }
    if (C->eps_blocks) {
        C->pair.scale = reinterpret_cast<const double*>(ws + C->o_pair_scale);
        C->pair.tile_block = reinterpret_cast<const int*>(ws + C->o_tile_block);
        for (int a = 0; a < 3; ++a) {
            C->pair.epb[a] = C->eps_epb[a];
            C->pair.nb[a] = C->eps_nb[a];
        }
    }
    if (!C->rec_ptr.empty()) {
        C->rec.ptr = reinterpret_cast<const int*>(ws + C->o_rec_ptr);
        C->rec.idx = reinterpret_cast<const int*>(ws + C->o_rec_idx);
        C->rec.val = reinterpret_cast<const double*>(ws + C->o_rec_val);
        C->rec.nrows = (int)C->rec_ptr.size() - 1;
    }
    // pairing sweeps
    for (int which = 0; which < 2; ++which) {
        const int fld = which == 0 ? SMX_FIELD_D : SMX_FIELD_B;
        for (int a = 0; a < 3; ++a) {
            SolveArgs& S = C->solve[which][a];
            S.field = C->fld[fld];
            S.axis = a;
            for (int c = 0; c < 3; ++c) {
                const int w = factor_index(which, c, a);
                S.f[c].L = reinterpret_cast<const double*>(ws + C->o_fac[a][w][0]);
                S.f[c].U = reinterpret_cast<const double*>(ws + C->o_fac[a][w][1]);
                S.f[c].dinv = reinterpret_cast<const double*>(ws + C->o_fac[a][w][2]);
                S.f[c].n = C->fac[a][w].n;
            }
        }
    }
    for (int h = 0; h < 2; ++h) {
        const HodgeHost& H = C->hodge[h];
        const int fld = kFieldOfHodge[h];
        if (H.mode == 0) {
            HodgeBlockArgs& A = C->hb[h];
            A.field = C->fld[fld];
            for (int a = 0; a < 3; ++a) {
                A.ntile[a] = H.ntile[a];
                A.tf0[a] = reinterpret_cast<const int*>(ws + H.o_tf0[a]);
                A.tlen[a] = reinterpret_cast<const int*>(ws + H.o_tlen[a]);
                A.tmat[a] = reinterpret_cast<const double*>(ws + H.o_tmat[a]);
            }
            for (int c = 0; c < 3; ++c)
                for (int a = 0; a < 3; ++a) {
                    A.kinds[c][a] = kFieldKinds[fld][c][a];
                    A.deg[c][a] = kind_degree(A.kinds[c][a], C->p[a]);
                }
            A.gamma = reinterpret_cast<const double*>(ws + H.o_gamma);
            A.max_nloc = H.max_nloc;
            if (H.separable) {
                const int which = h == 0 ? 1 : 0;  // M^2 pairs with K~_1, M~^2 with K_1
                for (int a = 0; a < 3; ++a) {
                    MassSolveArgs& M = C->ms[h][a];
                    M.field = C->fld[fld];
                    M.axis = a;
                    for (int c = 0; c < 3; ++c) {
                        const int kind = kFieldKinds[fld][c][a];
                        M.f[c] = C->solve[which][a].f[c];
                        M.mass[c] = reinterpret_cast<const double*>(ws + H.o_lmass[a][kind]);
                        M.deg[c] = kind_degree(kind, C->p[a]);
                    }
                }
            }
        } else {
            HodgeQuadArgs& A = C->hq[h];
            A.field = C->fld[fld];
            for (int a = 0; a < 3; ++a) {
                A.nel[a] = C->nel[a];
                A.q[a] = H.q[a];
                A.Qn[a] = H.Qn[a];
                A.bval[a] = reinterpret_cast<const double*>(ws + H.o_bval[a]);
            }
            for (int c = 0; c < 3; ++c)
                for (int a = 0; a < 3; ++a) {
                    A.kinds[c][a] = kFieldKinds[fld][c][a];
                    A.deg[c][a] = kind_degree(A.kinds[c][a], C->p[a]);
                    A.koff[c][a] = kind_offset(A.kinds[c][a]);
                }
            A.G = reinterpret_cast<const double*>(ws + H.o_G);
            A.Qtot = H.Qtot;
        }
    }
    if (C->use_digit)
        for (int h = 0; h < 2; ++h)
            for (int a = 0; a < 3; ++a) {
                const int fld = kFieldOfHodge[h];
                ModeDigitArgs& Mg = C->mdg[h][a];
                Mg.field = C->fld[fld];
                Mg.axis = a;
                Mg.status = C->status;
                for (int c = 0; c < 3; ++c) {
                    Mg.B[c] = static_cast<const void*>(ws + C->o_dig[h][a][c]);
                    Mg.rowexp[c] = reinterpret_cast<const int*>(ws + C->o_dige[h][a][c]);
                    Mg.npad[c] = mode_digit_npad(C->fld[fld].c[c].n[a]);
                }
            }
    if (C->s1) {
        for (int k = 0; k < 3; ++k) C->s1v[k] = reinterpret_cast<double*>(ws + C->o_s1v[k]);
        C->cg = reinterpret_cast<double*>(ws + C->o_cg);
        const int flds1[2] = {SMX_FIELD_H, SMX_FIELD_E};
        for (int k = 0; k < 2; ++k) {
            const HodgeHost& H = C->hodge1[k];
            const int fld = flds1[k];
            if (H.mode == 0) {
                HodgeBlockArgs& A = C->hb1[k];
                A.field = C->fld[fld];
                for (int a = 0; a < 3; ++a) {
                    A.ntile[a] = H.ntile[a];
                    A.tf0[a] = reinterpret_cast<const int*>(ws + H.o_tf0[a]);
                    A.tlen[a] = reinterpret_cast<const int*>(ws + H.o_tlen[a]);
                    A.tmat[a] = reinterpret_cast<const double*>(ws + H.o_tmat[a]);
                }
                for (int c = 0; c < 3; ++c)
                    for (int a = 0; a < 3; ++a) {
                        A.kinds[c][a] = kFieldKinds[fld][c][a];
                        A.deg[c][a] = kind_degree(A.kinds[c][a], C->p[a]);
                    }
                A.gamma = reinterpret_cast<const double*>(ws + H.o_gamma);
                A.max_nloc = H.max_nloc;
            } else {
                HodgeQuadArgs& Q = C->hq1[k];
                Q.field = C->fld[fld];
                for (int a = 0; a < 3; ++a) {
                    Q.nel[a] = C->nel[a];
                    Q.q[a] = H.q[a];
                    Q.Qn[a] = H.Qn[a];
                    Q.bval[a] = reinterpret_cast<const double*>(ws + H.o_bval[a]);
                }
                for (int c = 0; c < 3; ++c)
                    for (int a = 0; a < 3; ++a) {
                        Q.kinds[c][a] = kFieldKinds[fld][c][a];
                        Q.deg[c][a] = kind_degree(Q.kinds[c][a], C->p[a]);
                        Q.koff[c][a] = kind_offset(Q.kinds[c][a]);
                    }
                Q.G = reinterpret_cast<const double*>(ws + H.o_G);
                Q.Qtot = H.Qtot;
            }
            for (int a = 0; a < 3; ++a) {
                SolveArgs& S = C->pre1[k][a];
                S.field = C->fld[fld];
                S.axis = a;
                for (int c = 0; c < 3; ++c) {
                    const int kind = kFieldKinds[fld][c][a];
                    S.f[c].L = reinterpret_cast<const double*>(ws + C->o_mfac[a][kind][0]);
                    S.f[c].U = reinterpret_cast<const double*>(ws + C->o_mfac[a][kind][1]);
                    S.f[c].dinv = reinterpret_cast<const double*>(ws + C->o_mfac[a][kind][2]);
                    S.f[c].n = C->mfac[a][kind].n;
                }
                // K_2 = K~_1^T along the axis: the transposes of K~_1's factors (which = 1); K~_2 = K_1^T
                BandApplyArgs& Ba = C->kt[k][a];
                Ba.field = C->fld[fld];
                Ba.axis = a;
                Ba.kl = C->p[a] - 1;
                const int which = k == 0 ? 1 : 0;
                for (int c = 0; c < 3; ++c)
                    Ba.band[c] = reinterpret_cast<const double*>(ws + C->o_band[a][factor_index(which, c, a) ^ 2]);
            }
        }
    }
    if (C->precision == SMX_MIXED_REFINED) {
        for (int which = 0; which < 2; ++which) {
            const int fld = which == 0 ? SMX_FIELD_D : SMX_FIELD_B;
            for (int a = 0; a < 3; ++a) {
                LineF32Args& Lt = C->ln32T[which][a];
                BandApplyArgs& Bt = C->bandT[which][a];
                Lt.field = Bt.field = C->fld[fld];
                Lt.axis = Bt.axis = a;
                Bt.kl = C->p[a] - 1;
                for (int c = 0; c < 3; ++c) {
                    const int w = factor_index(which, c, a) ^ 2;  // the transposed factor
                    Lt.L[c] = reinterpret_cast<const float2*>(ws + C->o_fac32[a][w][0]);
                    Lt.U[c] = reinterpret_cast<const float2*>(ws + C->o_fac32[a][w][1]);
                    Lt.dinv[c] = reinterpret_cast<const float2*>(ws + C->o_fac32[a][w][2]);
                    Lt.mass[c] = nullptr;
                    Lt.deg[c] = 0;
                    Bt.band[c] = reinterpret_cast<const double*>(ws + C->o_band[a][w]);
                }
            }
        }
        C->t64 = reinterpret_cast<double*>(ws + C->o_t64);
        for (int h = 0; h < 2; ++h) {
            const int fld = kFieldOfHodge[h], which = h == 0 ? 1 : 0;  // M^2 pairs with K~_1, M~^2 with K_1
            for (int a = 0; a < 3; ++a) {
                BandApplyArgs& Ba = C->band[h][a];
                Ba.field = C->fld[fld];
                Ba.axis = a;
                Ba.kl = C->p[a] - 1;
                for (int c = 0; c < 3; ++c)
                    Ba.band[c] = reinterpret_cast<const double*>(ws + C->o_band[a][factor_index(which, c, a)]);
            }
        }
    }
    if (C->precision != SMX_FP64) {
        C->e32 = reinterpret_cast<float*>(ws + C->o_e32);
        C->h32 = reinterpret_cast<float*>(ws + C->o_h32);
        C->y32 = reinterpret_cast<float*>(ws + C->o_y32);
        for (int h = 0; h < 2; ++h) {
            const HodgeHost& H = C->hodge[h];
            const int fld = kFieldOfHodge[h];
            const int which = h == 0 ? 1 : 0;  // M^2 pairs with K~_1, M~^2 with K_1
            if (H.mode == 1) {
                HodgeQuadF32Args& Q = C->hq32[h];
                const HodgeQuadArgs& Q64 = C->hq[h];
                Q.field = Q64.field;
                for (int a = 0; a < 3; ++a) {
                    Q.nel[a] = Q64.nel[a];
                    Q.q[a] = Q64.q[a];
                    Q.Qn[a] = Q64.Qn[a];
                    Q.bval[a] = reinterpret_cast<const float2*>(ws + C->o_bval32[h][a]);
                    for (int c = 0; c < 3; ++c) {
                        Q.kinds[a][c] = Q64.kinds[a][c];
                        Q.deg[a][c] = Q64.deg[a][c];
                        Q.koff[a][c] = Q64.koff[a][c];
                    }
                }
                Q.G = reinterpret_cast<const float2*>(ws + C->o_G32[h]);
                Q.Qtot = Q64.Qtot;
            }
            HodgeBlockF32Args& B = C->hb32[h];
            B.field = C->fld[fld];
            B.compensated = C->precision == SMX_MIXED_REFINED ? 1 : 0;
            for (int a = 0; a < 3; ++a) {
                B.ntile[a] = H.ntile[a];
                B.tf0[a] = reinterpret_cast<const int*>(ws + H.o_tf0[a]);
                B.tlen[a] = reinterpret_cast<const int*>(ws + H.o_tlen[a]);
                B.tmat[a] = reinterpret_cast<const float2*>(ws + C->o_tmat32[h][a]);
            }
            for (int c = 0; c < 3; ++c)
                for (int a = 0; a < 3; ++a) {
                    B.kinds[c][a] = kFieldKinds[fld][c][a];
                    B.deg[c][a] = kind_degree(B.kinds[c][a], C->p[a]);
                }
            B.gamma = reinterpret_cast<const double*>(ws + H.o_gamma);
            B.max_nloc = H.max_nloc;
            for (int a = 0; a < 2; ++a) {
                int m = 1;
                for (int c = 0; c < 3; ++c)
                    for (int t = 0; t < H.ntile[a]; ++t)
                        m = std::max(m, H.tlen[a].empty() ? 1 : H.tlen[a][kFieldKinds[fld][c][a] * H.ntile[a] + t]);
                B.max_len[a] = m;
            }
            for (int a = 0; a < 3; ++a) {
                ModeF32Args& Md = C->md32[h][a];
                Md.field = C->fld[fld];
                Md.axis = a;
                for (int c = 0; c < 3; ++c)
                    Md.B[c] = C->use_mode ? reinterpret_cast<const float2*>(ws + C->o_mode32[h][a][c]) : nullptr;
                int maxn = 0;
                for (int c = 0; c < 3; ++c) maxn = std::max(maxn, C->fld[fld].c[c].n[a]);
                Md.npad = mode_f32_npad(maxn);
            }
            for (int a = 0; a < 3; ++a) {
                LineF32Args& Lg = C->ln32[h][a];
                Lg.field = C->fld[fld];
                Lg.axis = a;
                for (int c = 0; c < 3; ++c) {
                    const int w = factor_index(which, c, a), kind = kFieldKinds[fld][c][a];
                    Lg.L[c] = reinterpret_cast<const float2*>(ws + C->o_fac32[a][w][0]);
                    Lg.U[c] = reinterpret_cast<const float2*>(ws + C->o_fac32[a][w][1]);
                    Lg.dinv[c] = reinterpret_cast<const float2*>(ws + C->o_fac32[a][w][2]);
                    Lg.mass[c] = H.separable ? reinterpret_cast<const float2*>(ws + C->o_lmass32[h][a][kind]) : nullptr;
                    Lg.deg[c] = kind_degree(kind, C->p[a]);
                }
            }
        }
    }
    return SMX_OK;
}

#define NEED_WS(C)                      \
    do {                                \
        if (!(C)) return SMX_EINVAL;    \
        if (!(C)->ws) return SMX_ESTATE; \
    } while (0)

int smx_curl_primal(smx_ctx* C, const double* e, double* b, double alpha) {
    NEED_WS(C);
    if (!e || !b || !std::isfinite(alpha)) return SMX_EINVAL;
    return curl_primal_impl(C, e, b, alpha);
}

int smx_curl_dual(smx_ctx* C, const double* h, double* d, double alpha, const double* jhat, double s) {
    NEED_WS(C);
    if (!h || !d || !std::isfinite(alpha) || !std::isfinite(s)) return SMX_EINVAL;
    return curl_dual_impl(C, h, d, alpha, jhat, nullptr, 0, s);
}

int smx_hodge_apply(smx_ctx* C, int field, const double* x, double* y) {
    NEED_WS(C);
    if (!x || !y || x == y) return SMX_EINVAL;
    if (field != SMX_FIELD_B && field != SMX_FIELD_D) return SMX_EINVAL;
    return hodge_apply_impl(C, field == SMX_FIELD_B ? 0 : 1, x, y);
}

int smx_pairing_solve(smx_ctx* C, int which, const double* y, double* x) {
    NEED_WS(C);
    if (!x || !y) return SMX_EINVAL;
    if (which != SMX_FIELD_E && which != SMX_FIELD_H) return SMX_EINVAL;
    return solve_impl(C, which == SMX_FIELD_E ? 0 : 1, y, x);
}

int smx_hodge_star(smx_ctx* C, int field, const double* x, double* out) {
    NEED_WS(C);
    if (!x || !out) return SMX_EINVAL;
    if (field != SMX_FIELD_B && field != SMX_FIELD_D) return SMX_EINVAL;
    return hodge_star_impl(C, field == SMX_FIELD_B ? 0 : 1, x, out);
}

int smx_step(smx_ctx* C, double* d, double* b, double* e, double* h, const double* jhat, const double* amp,
             double dt, int nsteps) {
    NEED_WS(C);
    if (!d || !b || !e || !h || nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return SMX_EINVAL;
    if (jhat && !amp) return SMX_EINVAL;
    if (nsteps == 0) return SMX_OK;
    // Replay a captured CUDA graph of the whole call: one launch instead of about
    // ten per step.  Eager launches when per-kernel timing is on or the stream is
    // the legacy default stream (which cannot be captured).
    if (C->timing || C->stream == nullptr || !C->use_graphs) return step_eager(C, d, b, e, h, jhat, amp, dt, nsteps);
    GraphCache& G = C->graph;
    const void* key[6] = {d, b, e, h, jhat, amp};
    bool hit = G.exec != nullptr && G.dt == dt && G.nsteps == nsteps;
    for (int i = 0; i < 6 && hit; ++i) hit = G.key[i] == key[i];
    if (!hit) {
        if (G.exec) {
            cudaGraphExecDestroy(G.exec);
            G.exec = nullptr;
        }
        const long long before = C->launches;
        CK(cudaStreamBeginCapture(C->stream, cudaStreamCaptureModeThreadLocal));
        const int st = step_eager(C, d, b, e, h, jhat, amp, dt, nsteps);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(C->stream, &graph);
        if (st || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            C->launches = before;
            return st ? st : SMX_ECUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            G.exec = nullptr;
            C->launches = before;
            return SMX_ECUDA;
        }
        G.kernels = C->launches - before;
        C->launches = before;
        G.dt = dt;
        G.nsteps = nsteps;
        for (int i = 0; i < 6; ++i) G.key[i] = key[i];
    }
    CK(cudaGraphLaunch(G.exec, C->stream));
    C->launches += G.kernels;
    return SMX_OK;
}

int smx_scheme1_star(smx_ctx* C, int field, const double* x, double* out, double tol, int maxit, int* iters) {
    NEED_WS(C);
    if (!C->s1) return SMX_ESTATE;
    if (!x || !out || x == out || !(tol > 0.0) || maxit < 0) return SMX_EINVAL;
    if (field != SMX_FIELD_B && field != SMX_FIELD_D) return SMX_EINVAL;
    return s1_star(C, field == SMX_FIELD_B ? 0 : 1, x, out, tol, maxit, iters);
}

int smx_step_scheme1(smx_ctx* C, double* d, double* b, double* e, double* h, const double* jhat, const double* amp,
                     double dt, int nsteps, double tol, int maxit, int* max_iters) {
    NEED_WS(C);
    if (!C->s1) return SMX_ESTATE;
    if (!d || !b || !e || !h || nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt) || !(tol > 0.0) || maxit < 0)
        return SMX_EINVAL;
    if (jhat && !amp) return SMX_EINVAL;
    int worst = 0, it = 0, st;
    if ((st = curl_primal_impl(C, e, b, -0.5 * dt))) return st;
    for (int n = 0; n < nsteps; ++n) {
        if ((st = s1_star(C, 0, b, h, tol, maxit, &it))) return st;  // h = (M~^1_mu)^{-1} K_2 b
        worst = std::max(worst, it);
        if ((st = curl_dual_impl(C, h, d, dt, jhat, amp, n, 0.0))) return st;
        if ((st = s1_star(C, 1, d, e, tol, maxit, &it))) return st;  // e = (M^1_eps)^{-1} K~_2 d
        worst = std::max(worst, it);
        if ((st = curl_primal_impl(C, e, b, (n + 1 == nsteps) ? -0.5 * dt : -dt))) return st;
    }
    if (max_iters) *max_iters = worst;
    return SMX_OK;
}

int smx_energy_scheme1(smx_ctx* C, const double* d, const double* b, const double* e, const double* h,
                       double* out) {
    NEED_WS(C);
    if (!C->s1) return SMX_ESTATE;
    if (!d || !b || !e || !h || !out) return SMX_EINVAL;
    // E_h = 1/2 (e^T K~_2 d + h^T K_2 b) (Sec. 3.3, energy with pairing matrices)
    int st = s1_pair_t(C, 1, d, C->scratch, C->s1v[0], C->s1v[1]);
    if (st) return st;
    if ((st = dot_impl(C, e, C->scratch, C->N_e, 0))) return st;
    if ((st = s1_pair_t(C, 0, b, C->scratch, C->s1v[0], C->s1v[1]))) return st;
    if ((st = dot_impl(C, h, C->scratch, C->N_h, 1))) return st;
    double host[2];
    CK(cudaMemcpyAsync(host, C->dots, sizeof host, cudaMemcpyDeviceToHost, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    out[0] = 0.5 * (host[0] + host[1]);
    return std::isfinite(out[0]) ? SMX_OK : SMX_ENONFINITE;
}

int smx_cfl_scheme1(smx_ctx* C, int iters, double tol, double* v, double* w, double* t, double cg_tol, int cg_maxit,
                    double* dt_max) {
    NEED_WS(C);
    if (!C->s1) return SMX_ESTATE;
    if (!v || !w || !t || !dt_max || iters < 1 || !(tol >= 0.0) || !(cg_tol > 0.0)) return SMX_EINVAL;
    // lambda_max of T = D~^1 S_H D^1 S_E by power iteration in the inner product of K_1 S_E
    // (T is self-adjoint there); S_E, S_H the scheme-1 Hodge stars.  w holds S_E v, t holds
    // D^1 S_E v, then S_H of it, then T v in w.
    std::vector<double> v0(C->N_e);
    uint64_t state = 0x5eed5eedULL;
    for (auto& x : v0) x = (double)(splitmix64(state) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    CK(cudaMemcpyAsync(v, v0.data(), v0.size() * sizeof(double), cudaMemcpyHostToDevice, C->stream));
    double lam = 0.0, lam_old = 0.0;
    int it_cg = 0, st;
    // A x = K_1 S_E x = (K~_2)^T S_E x; the inner product needs only x^T K_1 S_E x = (K~_2 x)^T S_E x
    for (int it = 0; it < iters; ++it) {
        if ((st = s1_star(C, 1, v, w, cg_tol, cg_maxit, &it_cg))) return st;           // w = S_E v
        CK(cudaMemsetAsync(t, 0, C->N_h * sizeof(double), C->stream));
        if ((st = curl_primal_impl(C, w, t, 1.0))) return st;                           // t = D^1 S_E v
        if ((st = s1_pair_t(C, 1, v, C->scratch2, C->s1v[0], C->s1v[1]))) return st;   // K~_2 v
        if ((st = dot_impl(C, w, C->scratch2, C->N_e, 0))) return st;                   // den = v.A v
        if ((st = s1_star(C, 0, t, C->state, cg_tol, cg_maxit, &it_cg))) return st;   // S_H D^1 S_E v
        CK(cudaMemsetAsync(w, 0, C->N_e * sizeof(double), C->stream));
        if ((st = curl_dual_impl(C, C->state, w, 1.0, nullptr, nullptr, 0, 0.0))) return st;  // w = T v
        if ((st = s1_star(C, 1, w, t, cg_tol, cg_maxit, &it_cg))) return st;           // t = S_E T v (N_e <= len t)
        if ((st = s1_pair_t(C, 1, v, C->scratch2, C->s1v[0], C->s1v[1]))) return st;
        if ((st = dot_impl(C, t, C->scratch2, C->N_e, 1))) return st;                   // num = v.A T v
        if ((st = s1_pair_t(C, 1, w, C->scratch2, C->s1v[0], C->s1v[1]))) return st;
        if ((st = dot_impl(C, t, C->scratch2, C->N_e, 2))) return st;                   // |T v|_A^2
        double host[3];
        CK(cudaMemcpyAsync(host, C->dots, 3 * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
        CK(cudaStreamSynchronize(C->stream));
        if (!std::isfinite(host[0]) || !std::isfinite(host[1]) || !(host[2] > 0.0) || !(host[0] > 0.0))
            return SMX_ENONFINITE;
        lam = host[1] / host[0];
        const double sc = 1.0 / std::sqrt(host[2]);
        if ((st = run(C, 7, 1, [&] { return launch_scale_copy(w, v, sc, C->N_e, C->stream); }))) return st;
        if (it > 0 && std::fabs(lam - lam_old) <= tol * std::fabs(lam)) break;
        lam_old = lam;
    }
    if (!(lam > 0.0)) return SMX_ENONFINITE;
    *dt_max = 2.0 / std::sqrt(lam);
    return SMX_OK;
}

int smx_set_graphs(smx_ctx* C, int enable) {
    if (!C) return SMX_EINVAL;
    C->use_graphs = enable ? 1 : 0;
    return SMX_OK;
}

int smx_set_mode_kernel(smx_ctx* C, int which) {
    if (!C || (which != SMX_MODE_TENSOR && which != SMX_MODE_SIMT && which != SMX_MODE_AUTO)) return SMX_EINVAL;
    if (which != C->mode_kernel && C->graph.exec) {  // a captured step launches the other kernel
        cudaGraphExecDestroy(C->graph.exec);
        C->graph.exec = nullptr;
    }
    C->mode_kernel = which;
    return SMX_OK;
}

int smx_project(const smx_ctx* C, int field, smx_field_fn fn, void* user, double* coeffs) {
    if (!C || !fn || !coeffs || (field != SMX_FIELD_B && field != SMX_FIELD_D)) return SMX_EINVAL;
    try {
        int iters = 0;
        return l2_project_2form(C->p, C->nel, C->gmap, field, fn, user, coeffs, 1e-14, 500, &iters);
    } catch (const std::bad_alloc&) {
        return SMX_ENOMEM;
    }
}

int smx_mode_kernel(const smx_ctx* C, int* which) {
    if (!C || !which) return SMX_EINVAL;
    *which = C->use_digit ? C->mode_kernel : SMX_MODE_SIMT;
    if (*which == SMX_MODE_AUTO && C->use_mode) *which = mixed_tensor(C) ? SMX_MODE_TENSOR : SMX_MODE_SIMT;
    return SMX_OK;
}

int smx_device_status(smx_ctx* C) {
    NEED_WS(C);
    unsigned v = 0;
    CK(cudaMemcpyAsync(&v, C->status, sizeof v, cudaMemcpyDeviceToHost, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    if (v == 0) return SMX_OK;
    CK(cudaMemsetAsync(C->status, 0, sizeof(unsigned), C->stream));
    CK(cudaStreamSynchronize(C->stream));
    return SMX_ETIMEOUT;
}

int smx_hodge_star_mixed(smx_ctx* C, int field, const double* x, double* out) {
    NEED_WS(C);
    if (!x || !out) return SMX_EINVAL;
    if (field != SMX_FIELD_B && field != SMX_FIELD_D) return SMX_EINVAL;
    if (C->precision == SMX_FP64) return SMX_ESTATE;
    const int h = field == SMX_FIELD_B ? 0 : 1;
    if (C->precision == SMX_MIXED_REFINED) return star_refined(C, h, x, out, false);
    float* o32 = h == 0 ? C->h32 : C->e32;
    return hodge_star_f32_impl(C, h, x, o32, out);
}

int smx_energy(smx_ctx* C, const double* d, const double* b, const double* e, double dt, double out[2]) {
    NEED_WS(C);
    if (!d || !b || !out || !std::isfinite(dt)) return SMX_EINVAL;
    int st = hodge_apply_impl(C, 1, d, C->scratch);
    if (st) return st;
    st = dot_impl(C, d, C->scratch, C->N_e, 0);
    if (st) return st;
    st = hodge_apply_impl(C, 0, b, C->scratch);
    if (st) return st;
    st = dot_impl(C, b, C->scratch, C->N_h, 1);
    if (st) return st;
    double host[3] = {0.0, 0.0, 0.0};
    if (e) {
        // c = D^1 e into the second scratch vector, M c into the first
        CK(cudaMemsetAsync(C->scratch2, 0, C->N_h * sizeof(double), C->stream));
        if ((st = curl_primal_impl(C, e, C->scratch2, 1.0))) return st;
        if ((st = hodge_apply_impl(C, 0, C->scratch2, C->scratch))) return st;
        if ((st = dot_impl(C, C->scratch2, C->scratch, C->N_h, 2))) return st;
    }
    CK(cudaMemcpyAsync(host, C->dots, 3 * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    const double Eh = 0.5 * (host[0] + host[1]);
    out[0] = Eh;
    out[1] = e ? Eh - dt * dt / 8.0 * host[2] : Eh;
    if (!std::isfinite(out[0]) || !std::isfinite(out[1])) return SMX_ENONFINITE;
    return SMX_OK;
}

int smx_step_host(smx_ctx* C, double* d, double* b, double* e, double* h, const double* jhat, const double* amp,
                  double dt, int nsteps) {
    NEED_WS(C);
    if (!d || !b || !e || !h) return SMX_EINVAL;
    double* dd = C->state;
    double* ed = dd + C->N_e;
    double* bd = ed + C->N_e;
    double* hd = bd + C->N_h;
    const size_t se = C->N_e * sizeof(double), sh = C->N_h * sizeof(double);
    // on any error, no copy may still read or write the caller's host buffers after the return
    auto fail = [&](int st) {
        cudaStreamSynchronize(C->stream);
        return st;
    };
    auto copy = [&](void* dst, const void* src, size_t n, cudaMemcpyKind kind) {
        return cudaMemcpyAsync(dst, src, n, kind, C->stream) == cudaSuccess;
    };
    if (!copy(dd, d, se, cudaMemcpyHostToDevice) || !copy(ed, e, se, cudaMemcpyHostToDevice) ||
        !copy(bd, b, sh, cudaMemcpyHostToDevice))
        return fail(SMX_ECUDA);
    const int st = smx_step(C, dd, bd, ed, hd, jhat, amp, dt, nsteps);
    if (st) return fail(st);
    if (!copy(d, dd, se, cudaMemcpyDeviceToHost) || !copy(e, ed, se, cudaMemcpyDeviceToHost) ||
        !copy(b, bd, sh, cudaMemcpyDeviceToHost) || !copy(h, hd, sh, cudaMemcpyDeviceToHost))
        return fail(SMX_ECUDA);
    CK(cudaStreamSynchronize(C->stream));
    return SMX_OK;
}

int smx_launch_count(const smx_ctx* C, int64_t* n) {
    if (!C || !n) return SMX_EINVAL;
    *n = C->launches;
    return SMX_OK;
}

int smx_set_timing(smx_ctx* C, int enable) {
    if (!C) return SMX_EINVAL;
    C->timing = enable ? 1 : 0;
    return SMX_OK;
}

int smx_kernel_times(smx_ctx* C, double* ms, int64_t* counts) {
    if (!C || !ms || !counts) return SMX_EINVAL;
    for (int k = 0; k < SMX_NCLASS; ++k) {
        ms[k] = 0.0;
        counts[k] = 0;
    }
    int st = SMX_OK;
    if (!C->timed.empty() && cudaStreamSynchronize(C->stream) != cudaSuccess) st = SMX_ECUDA;
    for (auto& t : C->timed) {
        float el = 0.0f;
        if (st == SMX_OK && cudaEventElapsedTime(&el, t.a, t.b) == cudaSuccess) {
            ms[t.cls] += el;
            counts[t.cls] += 1;
        }
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    C->timed.clear();
    return st;
}

int smx_kernel_work(const smx_ctx* C, int cls, int field, double* flops, double* bytes) {
    if (!C || !flops || !bytes || field < 0 || field > 3) return SMX_EINVAL;
    const double Ne = (double)C->N_e, Nh = (double)C->N_h;
    const bool bside = (field == SMX_FIELD_B || field == SMX_FIELD_H);  // K~_1 / M^2 side
    const double N = bside ? Nh : Ne;
    switch (cls) {
        case 0:  // curl_primal: b += alpha D^1 e, 3 differences + 1 FMA per output
            if (!bside) return SMX_EINVAL;
            *flops = 5.0 * Nh;
            *bytes = 8.0 * (Ne + 2.0 * Nh);
            return SMX_OK;
        case 1:  // curl_dual (without source)
            if (bside) return SMX_EINVAL;
            *flops = 5.0 * Ne;
            *bytes = 8.0 * (Nh + 2.0 * Ne);
            return SMX_OK;
        case 2:
        case 3: {
            const int h = bside ? 0 : 1;
            const HodgeHost& H = C->hodge[h];
            if ((cls == 2) != (H.mode == 0)) return SMX_EINVAL;
            const int fld = kFieldOfHodge[h];
            double f = 0.0;
            if (H.mode == 0) {
                // per tile and component: 2 * (sum of band widths of each 1D pass x the other extents)
                for (int c = 0; c < 3; ++c) {
                    std::vector<double> band_sum[3], len[3];
                    for (int a = 0; a < 3; ++a) {
                        const int kind = kFieldKinds[fld][c][a], d = kind_degree(kind, C->p[a]);
                        for (int t = 0; t < H.ntile[a]; ++t) {
                            const int L = H.tlen[a][kind * H.ntile[a] + t];
                            double bs = 0.0;
                            for (int i = 0; i < L; ++i) bs += std::min(L - 1, i + d) - std::max(0, i - d) + 1;
                            band_sum[a].push_back(bs);
                            len[a].push_back(L);
                        }
                    }
                    for (int tz = 0; tz < H.ntile[2]; ++tz)
                        for (int ty = 0; ty < H.ntile[1]; ++ty)
                            for (int tx = 0; tx < H.ntile[0]; ++tx)
                                f += 2.0 * (band_sum[0][tx] * len[1][ty] * len[2][tz] +
                                            len[0][tx] * band_sum[1][ty] * len[2][tz] +
                                            len[0][tx] * len[1][ty] * band_sum[2][tz]);
                }
            } else {
                const double Qe = (double)H.q[0] * H.q[1] * H.q[2];
                const double nel = (double)C->nel[0] * C->nel[1] * C->nel[2];
                double per = 15.0 * Qe;
                for (int c = 0; c < 3; ++c) {
                    double r[3];
                    for (int a = 0; a < 3; ++a) r[a] = kind_degree(kFieldKinds[fld][c][a], C->p[a]) + 1;
                    per += 4.0 * (r[2] * r[1] * H.q[0] * r[0] + r[2] * H.q[1] * H.q[0] * r[1] + Qe * r[2]);
                }
                f = per * nel;
            }
            *flops = f;
            *bytes = 16.0 * N + (H.mode == 1 ? 48.0 * (double)H.Qtot : 0.0);
            return SMX_OK;
        }
        case 4:
        case 5:
        case 6: {  // one 1D sweep: forward 2 KL + backward 2 KL + 1 flops per entry
            const int kl = C->p[cls - 4] - 1;
            *flops = (4.0 * kl + 1.0) * N;
            *bytes = 16.0 * N;
            return SMX_OK;
        }
        case 8:
        case 9:
        case 10: {  // fused mass + solve sweep: 2 (2 deg + 1) + 4 KL + 1 flops per entry
            const int h = bside ? 0 : 1;
            if (!C->hodge[h].separable) return SMX_EINVAL;
            const int a = cls - 8, kl = C->p[a] - 1, fld = kFieldOfHodge[h];
            double f = 0.0;
            for (int c = 0; c < 3; ++c) {
                const DevComp& K = C->fld[fld].c[c];
                const double nc = (double)K.n[0] * K.n[1] * K.n[2];
                const int d = kind_degree(kFieldKinds[fld][c][a], C->p[a]);
                f += nc * (2.0 * (2 * d + 1) + 4.0 * kl + 1.0);
            }
            *flops = f;
            *bytes = 16.0 * N;
            return SMX_OK;
        }
        // mixed step: the method's flops as above (split products not counted twice);
        // bytes with FP32 intermediates and the FP64 state
        case 11:
        case 12: {
            const int st = smx_kernel_work(C, cls - 11, field, flops, bytes);
            if (st) return st;
            *bytes = cls == 11 ? 4.0 * Ne + 16.0 * Nh : 4.0 * Nh + 16.0 * Ne;
            return SMX_OK;
        }
        case 13: {
            const int st = smx_kernel_work(C, 2, field, flops, bytes);
            if (st) return st;
            *bytes = 12.0 * N;
            return SMX_OK;
        }
        case 14:
        case 15:
        case 16: {
            const int h = bside ? 0 : 1, a = cls - 14;
            const bool sep = C->hodge[h].separable;
            const int st = smx_kernel_work(C, sep ? 8 + a : 4 + a, field, flops, bytes);
            if (st) return st;
            if (C->use_mode) {  // dense mode product: 2 n flops per entry
                const DevField& F = C->fld[kFieldOfHodge[h]];
                double f = 0.0;
                for (int c = 0; c < 3; ++c)
                    f += 2.0 * F.c[c].n[a] * ((double)F.c[c].n[0] * F.c[c].n[1] * F.c[c].n[2]);
                *flops = f;
            }
            *bytes = (sep && a == 0 ? 12.0 : 8.0) * N;
            return SMX_OK;
        }
        case 17:
            *flops = 0.0;
            *bytes = 12.0 * N;
            return SMX_OK;
        case 24:
        case 25:
        case 26: {  // the mixed step's dense mode product on the tensor cores: as the CUDA-core one
            const int st = smx_kernel_work(C, cls - 10, field, flops, bytes);
            if (st) return st;
            if (!C->use_digit) return SMX_EINVAL;
            return SMX_OK;
        }
        case 21:
        case 22:
        case 23: {  // FP64 dense mode product on the tensor cores: 2 n flops per entry
            const int h = bside ? 0 : 1, a = cls - 21;
            if (!C->use_digit) return SMX_EINVAL;
            const DevField& F = C->fld[kFieldOfHodge[h]];
            double f = 0.0;
            for (int c = 0; c < 3; ++c) f += 2.0 * F.c[c].n[a] * ((double)F.c[c].n[0] * F.c[c].n[1] * F.c[c].n[2]);
            *flops = f;
            *bytes = 16.0 * N;
            return SMX_OK;
        }
        case 27: {  // refinement residual: one banded pass of 2 KL + 1 FMAs per entry (the mean over the axes)
            const int h = bside ? 0 : 1;
            if (C->precision != SMX_MIXED_REFINED) return SMX_EINVAL;
            const DevField& F = C->fld[kFieldOfHodge[h]];
            double f = 0.0;
            for (int a = 0; a < 3; ++a) f += 2.0 * (2 * (C->p[a] - 1) + 1) * (double)F.total;
            *flops = f / 3.0;
            *bytes = (12.0 + 16.0 / 3.0 + 8.0 / 3.0) * N;  // x0 FP32 or FP64 in, FP64 out, y once
            return SMX_OK;
        }
        case 18: {  // FP32 quadrature Hodge: the FP64 quadrature kernel's flops, FP32 metric
            const int st = smx_kernel_work(C, 3, field, flops, bytes);
            if (st) return st;
            *bytes = 12.0 * N + 24.0 * (double)C->hodge[bside ? 0 : 1].Qtot;
            return SMX_OK;
        }
        default:
            return SMX_EINVAL;
    }
}

// ---- reverse step, receivers, block material updates
int smx_receivers_set(smx_ctx* C, int n, const double* xhat) {
    if (!C || n < 0 || (n > 0 && !xhat)) return SMX_EINVAL;
    if (C->ws) return SMX_ESTATE;  // the receiver table is part of the workspace layout
    if (!C->rec_ptr.empty()) return SMX_ESTATE;
    for (int k = 0; k < 3 * n; ++k)
        if (!(xhat[k] >= 0.0 && xhat[k] <= 1.0)) return SMX_EINVAL;
    try {
        std::vector<int> ptr(1, 0), idx;
        std::vector<double> val;
        const DevField& E = C->fld[SMX_FIELD_E];
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < 3; ++c) {
                // the component's basis along each axis at the point: the d+1 functions of its element
                double v[3][16];
                int i0[3], dim[3], deg[3];
                for (int a = 0; a < 3; ++a) {
                    const int kind = kFieldKinds[SMX_FIELD_E][c][a], nel = C->nel[a];
                    const double x = xhat[3 * r + a];
                    const int e = std::min(nel - 1, (int)(x * nel));
                    local_basis(kind, C->p[a], nel, e, x, v[a]);
                    i0[a] = e + kind_offset(kind);
                    dim[a] = kind_dim(kind, C->p[a], nel);
                    deg[a] = kind_degree(kind, C->p[a]);
                }
                for (int k = 0; k <= deg[2]; ++k)
                    for (int j = 0; j <= deg[1]; ++j)
                        for (int i = 0; i <= deg[0]; ++i) {
                            const int gi = i0[0] + i, gj = i0[1] + j, gk = i0[2] + k;
                            if (gi < 0 || gi >= dim[0] || gj < 0 || gj >= dim[1] || gk < 0 || gk >= dim[2]) continue;
                            const double w = v[0][i] * v[1][j] * v[2][k];
                            if (w == 0.0) continue;
                            idx.push_back((int)(E.c[c].off + gi + (long long)E.c[c].n[0] * (gj + (long long)E.c[c].n[1] * gk)));
                            val.push_back(w);
                        }
                ptr.push_back((int)idx.size());
            }
        if (idx.empty()) {  // keep the tables non-empty
            idx.push_back(0);
            val.push_back(0.0);
        }
        C->rec_ptr = ptr;
        C->rec_idx = idx;
        C->rec_val = val;
        C->o_rec_ptr = C->blob.add(C->rec_ptr);
        C->o_rec_idx = C->blob.add(C->rec_idx);
        C->o_rec_val = C->blob.add(C->rec_val);
        layout(C);
    } catch (const std::bad_alloc&) {
        return SMX_ENOMEM;
    }
    return SMX_OK;
}

int smx_receivers_eval(smx_ctx* C, const double* e, double* out) {
    NEED_WS(C);
    if (!e || !out || C->rec_ptr.empty()) return SMX_EINVAL;
    return run(C, 20, 1, [&] { return launch_receivers_eval(C->rec, e, out, C->stream); });
}

int smx_receivers_adjoint(smx_ctx* C, const double* w, double alpha, double* ebar) {
    NEED_WS(C);
    if (!w || !ebar || C->rec_ptr.empty() || !std::isfinite(alpha)) return SMX_EINVAL;
    return run(C, 20, 1, [&] { return launch_receivers_adjoint(C->rec, w, alpha, ebar, C->stream); });
}

int smx_set_material_blocks(smx_ctx* C, int field, const double* values) {
    NEED_WS(C);
    if (field != SMX_FIELD_D || !values || !C->eps_blocks) return SMX_EINVAL;
    const size_t nb = C->eps_vals.size();
    for (size_t k = 0; k < nb; ++k)
        if (!finite_pos(values[k])) return SMX_EMAT;
    HodgeHost& H = C->hodge[1];
    std::vector<double> scale(nb);
    for (size_t k = 0; k < nb; ++k) scale[k] = -1.0 / values[k];
    // The host copy of the tables (the blob) changes with the workspace: a later
    // smx_bind_workspace and the no-alloc call upload the blob, not the workspace.
    unsigned char* blob = C->blob.bytes.data();
    if (H.mode == 0) {
        for (size_t t = 0; t < H.gamma.size(); ++t) H.gamma[t] = 1.0 / values[H.tile_block[t]];
        std::memcpy(blob + H.o_gamma, H.gamma.data(), H.gamma.size() * sizeof(double));
        CK(cudaMemcpyAsync(C->ws + H.o_gamma, H.gamma.data(), H.gamma.size() * sizeof(double), cudaMemcpyHostToDevice,
                           C->stream));
    } else {
        // the stored metric carries gamma = 1/eps: scale each block's points by eps_old / eps_new
        std::vector<double> ratio(nb);
        for (size_t k = 0; k < nb; ++k) ratio[k] = C->eps_vals[k] / values[k];
        CK(cudaMemcpyAsync(C->scratch, ratio.data(), nb * sizeof(double), cudaMemcpyHostToDevice, C->stream));
        float2* g32 = C->precision != SMX_FP64 ? reinterpret_cast<float2*>(C->ws + C->o_G32[1]) : nullptr;
        CK(launch_rescale_metric(reinterpret_cast<double*>(C->ws + H.o_G), g32, C->hq[1], C->eps_epb, C->eps_nb,
                                 C->scratch, C->stream));
        // the same products on the host copy (one FP64 multiply each, so the copies stay bit-identical)
        rescale_metric_host(C, ratio);
    }
    std::memcpy(blob + C->o_pair_scale, scale.data(), nb * sizeof(double));
    CK(cudaMemcpyAsync(C->ws + C->o_pair_scale, scale.data(), nb * sizeof(double), cudaMemcpyHostToDevice, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    C->eps_vals.assign(values, values + nb);
    C->uid = g_next_uid.fetch_add(1);  // tables changed: the no-alloc array no longer holds them
    return SMX_OK;
}

int smx_step_adjoint(smx_ctx* C, const double* d_n, const double* d_np1, double* dbar, double* bbar,
                     const double* ebar, const double* jhat, double dt, double* amp_bar, double* eps_bar) {
    NEED_WS(C);
    if (!d_n || !d_np1 || !dbar || !bbar || !(dt > 0.0) || !std::isfinite(dt)) return SMX_EINVAL;
    if (C->precision == SMX_MIXED) return SMX_ESTATE;  // FP64 or the refined mixed form
    if (eps_bar && !C->eps_blocks) return SMX_EINVAL;
    const double a = 0.5 * dt;
    double* A1 = C->scratch;
    double* A2 = C->scratch2;
    const size_t be = (size_t)C->N_e * sizeof(double), bh = (size_t)C->N_h * sizeof(double);
    int st;
    // w = dbar + S_E^T (-a D^1^T bbar), with D^1^T = D~^1; eps pair (z1, d_{n+1})
    CK(cudaMemsetAsync(A1, 0, be, C->stream));
    if ((st = curl_dual_impl(C, bbar, A1, -a, nullptr, nullptr, 0, 0.0))) return st;
    if ((st = solveT_any(C, 0, A1, A2))) return st;
    if (eps_bar && (st = pair_impl(C, A2, d_np1, eps_bar))) return st;
    if ((st = mass_acc_any(C, 1, A2, dbar))) return st;
    // source amplitude: sbar_n = -dt jhat^T w
    if (jhat && amp_bar) {
        if ((st = run(C, 7, 2, [&] { return launch_dot(jhat, dbar, C->N_e, C->partial, amp_bar, C->stream); })))
            return st;
        if ((st = run(C, 20, 1, [&] { return launch_scale_copy(amp_bar, amp_bar, -dt, 1, C->stream); }))) return st;
    }
    // bbar' = bbar + dt S_H^T D~^1^T w, with D~^1^T = D^1
    CK(cudaMemsetAsync(A1, 0, bh, C->stream));
    if ((st = curl_primal_impl(C, dbar, A1, dt))) return st;
    if ((st = solveT_any(C, 1, A1, A2))) return st;
    if ((st = mass_acc_any(C, 0, A2, bbar))) return st;
    // dbar_n = w + S_E^T (-a D~^1 bbar' + ebar); eps pair (z3, d_n)
    CK(cudaMemsetAsync(A1, 0, be, C->stream));
    if ((st = curl_dual_impl(C, bbar, A1, -a, nullptr, nullptr, 0, 0.0))) return st;
    if (ebar && (st = run(C, 20, 1, [&] { return launch_axpy(ebar, A1, 1.0, C->N_e, C->stream); }))) return st;
    if ((st = solveT_any(C, 0, A1, A2))) return st;
    if (eps_bar && (st = pair_impl(C, A2, d_n, eps_bar))) return st;
    return mass_acc_any(C, 1, A2, dbar);
}

int smx_adjoint_terminal(smx_ctx* C, const double* d_N, const double* ebar, double* dbar, double* eps_bar) {
    NEED_WS(C);
    if (!d_N || !ebar || !dbar) return SMX_EINVAL;
    if (C->precision == SMX_MIXED) return SMX_ESTATE;  // FP64 or the refined mixed form
    if (eps_bar && !C->eps_blocks) return SMX_EINVAL;
    int st;
    if ((st = solveT_any(C, 0, ebar, C->scratch2))) return st;
    if (eps_bar && (st = pair_impl(C, C->scratch2, d_N, eps_bar))) return st;
    CK(cudaMemsetAsync(dbar, 0, (size_t)C->N_e * sizeof(double), C->stream));
    return mass_acc_any(C, 1, C->scratch2, dbar);
}

// ---- batched cavities
struct smx_batch {
    std::vector<smx_ctx*> ctx;
    bool refined = false;               // refined mixed contexts (else FP64)
    std::vector<BatchCavity> cav;       // FP64 step
    std::vector<BatchRefCavity> rcav;   // refined mixed step
    std::vector<int2> items[kRefPhases];
    size_t o_cav = 0, o_items[kRefPhases] = {}, o_bar = 0, o_status = 0, o_stepctr = 0, total = 0;
    size_t max_mass_floats = 0;         // largest FP32 mass unit (refined)
    int nphases() const { return refined ? kRefPhases : kBatchPhases; }
    unsigned char* ws = nullptr;
    cudaStream_t stream = nullptr;
    int maxn = 0, maxkl = 0, max_nloc = 0;
    size_t max_quad = 0;  // shared memory (doubles) of the largest quadrature element
    int line_warps = 0, grid = 0;
    size_t smem = 0;
    long long steps = 0;  // amplitude index of the next step (host mirror of the device counter)
    bool state_set = false;
    unsigned long long wait_ns = 1000000000ull;  // grid-barrier wait limit
    // captured CUDA graph of the last smx_batch_step call's nsteps launches
    int use_graphs = 1;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    ~smx_batch() {
        if (graph) cudaGraphExecDestroy(graph);
    }
    void drop_graph() {
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
    }
};

namespace {

void batch_curl_items(std::vector<int2>& list, int cav, const DevField& out) {
    int plane = 0, nz = 0;
    for (int c = 0; c < 3; ++c) {
        plane = std::max(plane, out.c[c].n[0] * out.c[c].n[1]);
        nz = std::max(nz, out.c[c].n[2]);
    }
    const int pb = (plane + kCurlThreads - 1) / kCurlThreads, zc = (nz + kCurlKz - 1) / kCurlKz;
    for (int c = 0; c < 3; ++c)
        for (int z = 0; z < zc; ++z)
            for (int b = 0; b < pb; ++b) list.push_back(make_int2(cav, batch_curl_unit(c, b, z)));
}

void batch_line_items(std::vector<int2>& list, int cav, const DevField& f, int axis) {
    for (int c = 0; c < 3; ++c) {
        const int n = f.c[c].n[axis];
        if (n <= 0) continue;
        const long long lines = (long long)f.c[c].n[0] * f.c[c].n[1] * f.c[c].n[2] / n;
        for (long long lb = 0; lb < (lines + kSolveLines - 1) / kSolveLines; ++lb)
            list.push_back(make_int2(cav, batch_comp_unit(c, (int)lb)));
    }
}

}  // namespace

// One refined mixed cavity: its tables and buffers (those of the single-cavity refined
// step) and its units in the twenty-five phases.
static void batch_refined_cavity(smx_batch* B, smx_ctx* C, int i) {
    BatchRefCavity K{};
    K.fE = C->fld[SMX_FIELD_E];
    K.fB = C->fld[SMX_FIELD_B];
    K.fH = C->fld[SMX_FIELD_H];
    K.fD = C->fld[SMX_FIELD_D];
    for (int h = 0; h < 2; ++h) {
        const HodgeHost& H = C->hodge[h];
        K.fS[h] = C->fld[kFieldOfHodge[h]];
        K.hb[h] = C->hb32[h];
        K.hq[h] = C->hq32[h];
        K.mode[h] = H.mode;
        for (int a = 0; a < 3; ++a) {
            K.ln[h][a] = C->ln32[h][a];
            K.band[h][a] = C->band[h][a];
        }
        B->max_mass_floats = std::max(B->max_mass_floats,
                                      H.mode == 0 ? batch_ref_mass_floats(H.max_nloc, 0, 0, 0)
                                                  : batch_ref_mass_floats(0, H.q[0], H.q[1], H.q[2]));
    }
    for (int a = 0; a < 3; ++a) {
        K.kl[a] = C->p[a] - 1;
        B->maxkl = std::max(B->maxkl, C->p[a] - 1);
        for (int c = 0; c < 3; ++c)
            for (int f = 0; f < 4; ++f) B->maxn = std::max(B->maxn, C->fld[f].c[c].n[a]);
    }
    K.y = C->scratch;
    K.t64 = C->t64;
    K.s64 = C->scratch2;
    K.x0[0] = C->h32;
    K.x0[1] = C->e32;
    K.c32 = C->y32;
    B->rcav.push_back(K);
    auto chunks = [&](int ph, long long ntot) {
        for (long long z = 0; z < (ntot + kBatchThreads * 8 - 1) / (kBatchThreads * 8); ++z)
            B->items[ph].push_back(make_int2(i, (int)z));
    };
    auto zeros = [&](int ph, long long ntot) {
        for (long long z = 0; z < (ntot + kBatchThreads * 8 - 1) / (kBatchThreads * 8); ++z)
            B->items[ph].push_back(make_int2(i, batch_zero_unit((int)z)));
    };
    batch_curl_items(B->items[0], i, K.fB);
    batch_curl_items(B->items[12], i, K.fD);
    batch_curl_items(B->items[24], i, K.fB);
    for (int h = 0; h < 2; ++h) {
        const int base = 12 * h;
        const HodgeHost& H = C->hodge[h];
        zeros(base, K.fS[h].total);
        if (H.mode == 0) {
            const int nt = H.ntile[0] * H.ntile[1] * H.ntile[2];
            for (int c = 0; c < 3; ++c)
                for (int t = 0; t < nt; ++t) B->items[base + 1].push_back(make_int2(i, batch_comp_unit(c, t)));
        } else {
            const int ne = C->nel[0] * C->nel[1] * C->nel[2];
            for (int e = 0; e < ne; ++e) B->items[base + 1].push_back(make_int2(i, e));
        }
        for (int a = 0; a < 3; ++a) {
            batch_line_items(B->items[base + 2 + a], i, K.fS[h], a);
            chunks(base + 5 + a, K.fS[h].total);
            batch_line_items(B->items[base + 8 + a], i, K.fS[h], a);
        }
        chunks(base + 11, K.fS[h].total);
    }
}

int smx_batch_create(int n, smx_ctx* const* ctxs, smx_batch** out) {
    if (n < 1 || !ctxs || !out) return SMX_EINVAL;
    *out = nullptr;
    smx_batch* B = new (std::nothrow) smx_batch();
    if (!B) return SMX_ENOMEM;
    B->refined = ctxs[0] && ctxs[0]->precision == SMX_MIXED_REFINED;
    try {
        for (int i = 0; i < n; ++i) {
            smx_ctx* C = ctxs[i];
            // bound, all FP64 or all refined mixed; any map and material
            if (!C || !C->ws || C->precision != (B->refined ? SMX_MIXED_REFINED : SMX_FP64)) {
                delete B;
                return SMX_EINVAL;
            }
            B->ctx.push_back(C);
            if (B->refined) {
                batch_refined_cavity(B, C, i);
                continue;
            }
            BatchCavity K{};
            K.fE = C->fld[SMX_FIELD_E];
            K.fB = C->fld[SMX_FIELD_B];
            K.fH = C->fld[SMX_FIELD_H];
            K.fD = C->fld[SMX_FIELD_D];
            for (int a = 0; a < 3; ++a) {
                K.msH[a] = C->ms[0][a];
                K.msD[a] = C->ms[1][a];
                K.solveH[a] = C->solve[1][a];
                K.solveE[a] = C->solve[0][a];
                K.kl[a] = C->p[a] - 1;
                B->maxkl = std::max(B->maxkl, C->p[a] - 1);
                for (int c = 0; c < 3; ++c)
                    for (int f = 0; f < 4; ++f) B->maxn = std::max(B->maxn, C->fld[f].c[c].n[a]);
            }
            K.hbB = C->hb[0];
            K.hbD = C->hb[1];
            K.hqB = C->hq[0];
            K.hqD = C->hq[1];
            K.sepB = C->hodge[0].separable ? 1 : 0;
            K.sepD = C->hodge[1].separable ? 1 : 0;
            K.modeB = C->hodge[0].mode;
            K.modeD = C->hodge[1].mode;
            K.y = C->scratch;
            for (int h = 0; h < 2; ++h) {
                const HodgeHost& H = C->hodge[h];
                if (H.mode == 0) B->max_nloc = std::max(B->max_nloc, H.max_nloc);
                else B->max_quad = std::max(B->max_quad, hodge_quad_smem_doubles(H.q[0], H.q[1], H.q[2]));
            }
            B->cav.push_back(K);
            // the mass apply of a star that is not fused: zero y in the curl phase before it, then
            // one unit per (component, tile) or per element
            auto mass_items = [&](int h, int zero_phase, int mass_phase, long long ntot) {
                const HodgeHost& H = C->hodge[h];
                const long long nz = (ntot + kBatchThreads * 8 - 1) / (kBatchThreads * 8);
                for (long long z = 0; z < nz; ++z) B->items[zero_phase].push_back(make_int2(i, batch_zero_unit((int)z)));
                if (H.mode == 0) {
                    const int nt = H.ntile[0] * H.ntile[1] * H.ntile[2];
                    for (int c = 0; c < 3; ++c)
                        for (int t = 0; t < nt; ++t) B->items[mass_phase].push_back(make_int2(i, batch_comp_unit(c, t)));
                } else {
                    const int ne = C->nel[0] * C->nel[1] * C->nel[2];
                    for (int e = 0; e < ne; ++e) B->items[mass_phase].push_back(make_int2(i, e));
                }
            };
            batch_curl_items(B->items[0], i, K.fB);
            batch_curl_items(B->items[10], i, K.fB);
            if (!K.sepB) mass_items(0, 0, 1, K.fB.total);
            for (int a = 0; a < 3; ++a) batch_line_items(B->items[2 + a], i, K.fH, a);
            batch_curl_items(B->items[5], i, K.fD);
            if (!K.sepD) mass_items(1, 5, 6, K.fD.total);
            for (int a = 0; a < 3; ++a) batch_line_items(B->items[7 + a], i, K.fD, a);
        }
        // workspace: cavity table, item lists, barrier and status words
        size_t off = 0;
        auto take = [&](size_t bytes) {
            const size_t o = off;
            off += (bytes + 255) & ~size_t(255);
            return o;
        };
        B->o_cav = take(B->refined ? B->rcav.size() * sizeof(BatchRefCavity) : B->cav.size() * sizeof(BatchCavity));
        for (int ph = 0; ph < B->nphases(); ++ph)
            B->o_items[ph] = take(std::max<size_t>(1, B->items[ph].size()) * sizeof(int2));
        B->o_bar = take(2 * sizeof(unsigned));
        B->o_status = take(sizeof(unsigned));
        B->o_stepctr = take(sizeof(unsigned));
        B->total = off;
    } catch (const std::bad_alloc&) {
        delete B;
        return SMX_ENOMEM;
    }
    *out = B;
    return SMX_OK;
}

int smx_batch_destroy(smx_batch* B) {
    delete B;
    return SMX_OK;
}

int smx_batch_workspace_bytes(const smx_batch* B, size_t* bytes) {
    if (!B || !bytes) return SMX_EINVAL;
    *bytes = B->total;
    return SMX_OK;
}

static int batch_configure(smx_batch* B, int line_warps) {
    size_t smem;
    if (B->refined) {
        const size_t warp = batch_ref_line_warp_floats(B->maxn, std::max(1, B->maxkl));
        smem = std::max(warp * line_warps, B->max_mass_floats) * sizeof(float);
    } else {
        const size_t warp = batch_line_warp_doubles(B->maxn, std::max(1, B->maxkl));
        const size_t hodge = std::max((size_t)3 * kLMax * (kLMax + 1) + 2 * (size_t)B->max_nloc + 8, B->max_quad);
        smem = std::max(warp * line_warps, hodge) * sizeof(double);
    }
    if (smem > 226 * 1024) return SMX_EINVAL;
    const int per_sm = B->refined ? batch_refined_blocks_per_sm(smem) : batch_blocks_per_sm(smem);
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) return SMX_EINVAL;
    if (B->line_warps != line_warps || B->smem != smem || B->grid != per_sm * sms) B->drop_graph();
    B->line_warps = line_warps;
    B->smem = smem;
    B->grid = per_sm * sms;
    return SMX_OK;
}

int smx_batch_bind_workspace(smx_batch* B, void* dev, size_t bytes) {
    if (!B || !dev) return SMX_EINVAL;
    if (bytes < B->total || (reinterpret_cast<uintptr_t>(dev) & 255)) return SMX_ESTATE;
    B->ws = static_cast<unsigned char*>(dev);
    B->stream = B->ctx[0]->stream;
    for (int ph = 0; ph < B->nphases(); ++ph)
        if (!B->items[ph].empty())
            CK(cudaMemcpyAsync(B->ws + B->o_items[ph], B->items[ph].data(), B->items[ph].size() * sizeof(int2),
                               cudaMemcpyHostToDevice, B->stream));
    CK(cudaMemsetAsync(B->ws + B->o_bar, 0, 2 * sizeof(unsigned) + 256, B->stream));
    CK(cudaStreamSynchronize(B->stream));
    // default: as many line warps as the shared memory allows, at most 8
    int lw = 8;
    while (lw > 1 && batch_configure(B, lw) != SMX_OK) --lw;
    return batch_configure(B, lw);
}

int smx_batch_set_state(smx_batch* B, int i, double* d, double* b, double* e, double* h, const double* jhat,
                        const double* amp, double dt) {
    if (!B || !B->ws || i < 0 || i >= (int)B->ctx.size() || !d || !b || !e || !h) return SMX_EINVAL;
    if (!(dt > 0.0) || !std::isfinite(dt) || (jhat && !amp)) return SMX_EINVAL;
    if (B->refined) {
        BatchRefCavity& K = B->rcav[i];
        K.d = d;
        K.b = b;
        K.e = e;
        K.h = h;
        K.jhat = jhat;
        K.amp = amp;
        K.dt = dt;
        B->state_set = false;
        B->steps = 0;
        return SMX_OK;
    }
    BatchCavity& K = B->cav[i];
    K.d = d;
    K.b = b;
    K.e = e;
    K.h = h;
    K.jhat = jhat;
    K.amp = amp;
    K.dt = dt;
    B->state_set = false;
    B->steps = 0;
    return SMX_OK;
}

static int batch_launch(smx_batch* B, int nsteps) {
    if (!B->state_set) {
        if (B->refined) {
            for (const BatchRefCavity& K : B->rcav)
                if (!K.d) return SMX_ESTATE;
            CK(cudaMemcpyAsync(B->ws + B->o_cav, B->rcav.data(), B->rcav.size() * sizeof(BatchRefCavity),
                               cudaMemcpyHostToDevice, B->stream));
        } else {
            for (const BatchCavity& K : B->cav)
                if (!K.d) return SMX_ESTATE;
            CK(cudaMemcpyAsync(B->ws + B->o_cav, B->cav.data(), B->cav.size() * sizeof(BatchCavity),
                               cudaMemcpyHostToDevice, B->stream));
        }
        const unsigned ctr = (unsigned)B->steps;  // the device step counter follows the host's
        CK(cudaMemcpyAsync(B->ws + B->o_stepctr, &ctr, sizeof ctr, cudaMemcpyHostToDevice, B->stream));
        CK(cudaStreamSynchronize(B->stream));   // ctr is a stack variable
        B->state_set = true;
    }
    BatchArgs A{};
    BatchRefArgs R{};
    if (B->refined) {
        R.cav = reinterpret_cast<const BatchRefCavity*>(B->ws + B->o_cav);
        for (int ph = 0; ph < kRefPhases; ++ph) {
            R.items[ph] = reinterpret_cast<const int2*>(B->ws + B->o_items[ph]);
            R.nitems[ph] = (int)B->items[ph].size();
        }
        R.bar = reinterpret_cast<unsigned*>(B->ws + B->o_bar);
        R.status = reinterpret_cast<unsigned*>(B->ws + B->o_status);
        R.stepctr = reinterpret_cast<unsigned*>(B->ws + B->o_stepctr);
        R.line_warps = B->line_warps;
        R.warp_floats = (int)batch_ref_line_warp_floats(B->maxn, std::max(1, B->maxkl));
        R.wait_ns = B->wait_ns;
    } else {
        A.cav = reinterpret_cast<const BatchCavity*>(B->ws + B->o_cav);
        for (int ph = 0; ph < kBatchPhases; ++ph) {
            A.items[ph] = reinterpret_cast<const int2*>(B->ws + B->o_items[ph]);
            A.nitems[ph] = (int)B->items[ph].size();
        }
        A.bar = reinterpret_cast<unsigned*>(B->ws + B->o_bar);
        A.status = reinterpret_cast<unsigned*>(B->ws + B->o_status);
        A.stepctr = reinterpret_cast<unsigned*>(B->ws + B->o_stepctr);
        A.line_warps = B->line_warps;
        A.warp_smem = (int)batch_line_warp_doubles(B->maxn, std::max(1, B->maxkl));
        A.wait_ns = B->wait_ns;
    }
    auto launch_one = [&]() {
        return B->refined ? launch_batch_refined_step(R, B->grid, B->smem, B->stream)
                          : launch_batch_step(A, B->grid, B->smem, B->stream);
    };
    // the nsteps launches as one captured CUDA graph (replayed while nsteps and the shape are
    // unchanged; the step index comes from the device counter), eagerly on the legacy stream
    if (B->use_graphs && B->stream != nullptr && nsteps > 0) {
        if (!B->graph || B->graph_steps != nsteps) {
            B->drop_graph();
            CK(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t el = cudaSuccess;
            for (int n = 0; n < nsteps && el == cudaSuccess; ++n) el = launch_one();
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(B->stream, &g);
            if (el != cudaSuccess || ec != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return SMX_ECUDA;
            }
            const cudaError_t ei = cudaGraphInstantiate(&B->graph, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                B->graph = nullptr;
                return SMX_ECUDA;
            }
            B->graph_steps = nsteps;
        }
        CK(cudaGraphLaunch(B->graph, B->stream));
        B->steps += nsteps;
        return SMX_OK;
    }
    for (int n = 0; n < nsteps; ++n) {
        CK(launch_one());
        ++B->steps;
    }
    return SMX_OK;
}

int smx_batch_set_graphs(smx_batch* B, int enable) {
    if (!B) return SMX_EINVAL;
    B->use_graphs = enable ? 1 : 0;
    if (!enable) B->drop_graph();
    return SMX_OK;
}

int smx_batch_step(smx_batch* B, int nsteps) {
    if (!B || !B->ws || nsteps < 0) return SMX_EINVAL;
    return batch_launch(B, nsteps);
}

int smx_batch_status(smx_batch* B) {
    if (!B || !B->ws) return SMX_EINVAL;
    unsigned v = 0;
    CK(cudaMemcpyAsync(&v, B->ws + B->o_status, sizeof v, cudaMemcpyDeviceToHost, B->stream));
    CK(cudaStreamSynchronize(B->stream));
    if (v == 0) return SMX_OK;
    CK(cudaMemsetAsync(B->ws + B->o_status, 0, sizeof(unsigned), B->stream));
    CK(cudaMemsetAsync(B->ws + B->o_bar, 0, 2 * sizeof(unsigned), B->stream));
    CK(cudaStreamSynchronize(B->stream));
    return SMX_ETIMEOUT;
}

int smx_batch_set_wait_limit(smx_batch* B, double seconds) {
    if (!B || !(seconds >= 0.0) || seconds > 60.0) return SMX_EINVAL;
    B->drop_graph();  // the limit is a launch parameter of the captured launches
    B->wait_ns = (unsigned long long)(seconds * 1e9);
    return SMX_OK;
}

int smx_batch_autotune(smx_batch* B, int steps, int* line_warps) {
    if (!B || !B->ws || steps < 1) return SMX_EINVAL;
    // time each shape on the contexts' own state vectors (zero fields: the work does not depend on the data)
    std::vector<BatchCavity> saved = B->cav;
    std::vector<BatchRefCavity> rsaved = B->rcav;
    const long long saved_steps = B->steps;
    for (size_t i = 0; i < B->ctx.size(); ++i) {
        smx_ctx* C = B->ctx[i];
        double* d = C->state;
        double* e = C->state + C->N_e;
        double* b = C->state + 2 * C->N_e;
        double* h = b + C->N_h;
        if (B->refined) {
            BatchRefCavity& K = B->rcav[i];
            K.d = d;
            K.e = e;
            K.b = b;
            K.h = h;
            K.jhat = nullptr;
            K.amp = nullptr;
            K.dt = 1e-3;
        } else {
            BatchCavity& K = B->cav[i];
            K.d = d;
            K.e = e;
            K.b = b;
            K.h = h;
            K.jhat = nullptr;
            K.amp = nullptr;
            K.dt = 1e-3;
        }
        CK(cudaMemsetAsync(C->state, 0, 2 * (size_t)(C->N_e + C->N_h) * sizeof(double), C->stream));
    }
    B->state_set = false;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_lw = B->line_warps;
    for (int lw = 1; lw <= 8; lw *= 2) {
        if (batch_configure(B, lw) != SMX_OK) continue;
        int st = batch_launch(B, 1);  // warm-up
        if (st) return st;
        CK(cudaEventRecord(e0, B->stream));
        if ((st = batch_launch(B, steps))) return st;
        CK(cudaEventRecord(e1, B->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            best_lw = lw;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->cav = saved;
    B->rcav = rsaved;
    B->steps = saved_steps;
    B->state_set = false;
    const int st = batch_configure(B, best_lw);
    if (line_warps) *line_warps = best_lw;
    return st;
}

int smx_hodge_star_noalloc(smx_ctx* C, int field, const double* x, double* out) {
    if (!C || !x || !out) return SMX_EINVAL;
    if (field != SMX_FIELD_B && field != SMX_FIELD_D) return SMX_EINVAL;
    const int h = field == SMX_FIELD_B ? 0 : 1;
    const HodgeHost& H = C->hodge[h];
    if (H.mode != 0) return SMX_EINVAL;  // quadrature tables do not fit the fixed array
    const int fld = kFieldOfHodge[h];
    const long long n = C->fld[fld].total;
    // layout of the fixed array: this context's tables (as in the workspace), then one vector
    const size_t o_y = C->tables_bytes;
    if (o_y + (size_t)n * sizeof(double) > (size_t)SMX_NOALLOC_BYTES) return SMX_ENOSPACE;
    // the array is looked up for the current device; the kernels run on the context stream
    if (C->stream) {
        int cur = 0, sdev = 0;
        CK(cudaGetDevice(&cur));
        CK(cudaStreamGetDevice(C->stream, &sdev));
        if (cur != sdev) return SMX_EINVAL;
    }
    void* basev = nullptr;
    uint64_t* owner = nullptr;
    const int st = noalloc_region(&basev, &owner);
    if (st) return st;
    unsigned char* base = static_cast<unsigned char*>(basev);
    if (*owner != C->uid) {
        CK(cudaMemcpyAsync(base, C->blob.bytes.data(), C->blob.bytes.size(), cudaMemcpyHostToDevice, C->stream));
        *owner = C->uid;
    }
    HodgeBlockArgs A;
    A.field = C->fld[fld];
    for (int a = 0; a < 3; ++a) {
        A.ntile[a] = H.ntile[a];
        A.tf0[a] = reinterpret_cast<const int*>(base + H.o_tf0[a]);
        A.tlen[a] = reinterpret_cast<const int*>(base + H.o_tlen[a]);
        A.tmat[a] = reinterpret_cast<const double*>(base + H.o_tmat[a]);
    }
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a) {
            A.kinds[c][a] = kFieldKinds[fld][c][a];
            A.deg[c][a] = kind_degree(A.kinds[c][a], C->p[a]);
        }
    A.gamma = reinterpret_cast<const double*>(base + H.o_gamma);
    A.max_nloc = H.max_nloc;
    const int which = h == 0 ? 1 : 0;  // M^2 -> K~_1 solve, M~^2 -> K_1 solve
    SolveArgs S[3];
    for (int a = 0; a < 3; ++a) {
        S[a].field = C->fld[which == 0 ? SMX_FIELD_D : SMX_FIELD_B];
        S[a].axis = a;
        for (int c = 0; c < 3; ++c) {
            const int w = factor_index(which, c, a);
            S[a].f[c].L = reinterpret_cast<const double*>(base + C->o_fac[a][w][0]);
            S[a].f[c].U = reinterpret_cast<const double*>(base + C->o_fac[a][w][1]);
            S[a].f[c].dinv = reinterpret_cast<const double*>(base + C->o_fac[a][w][2]);
            S[a].f[c].n = C->fac[a][w].n;
        }
    }
    double* y = reinterpret_cast<double*>(base + o_y);
    CK(cudaMemsetAsync(y, 0, (size_t)n * sizeof(double), C->stream));  // the mass apply accumulates
    CK(launch_hodge_block(A, x, y, C->stream));
    CK(launch_solve_axis(S[0], C->p[0] - 1, y, out, C->stream));
    CK(launch_solve_axis(S[1], C->p[1] - 1, out, out, C->stream));
    CK(launch_solve_axis(S[2], C->p[2] - 1, out, out, C->stream));
    return SMX_OK;
}

int smx_factor_matrix(const smx_ctx* C, int axis, int which, int64_t* n, double* dense_out) {
    if (!C || !n || axis < 0 || axis > 2 || which < 0 || which > 3) return SMX_EINVAL;
    const BandLU& f = C->fac[axis][which];
    *n = f.n;
    if (dense_out) {
        const std::vector<double> A = band_lu_dense(f);
        std::memcpy(dense_out, A.data(), A.size() * sizeof(double));
    }
    return SMX_OK;
}

int smx_hodge_mode(const smx_ctx* C, int field, int* mode) {
    if (!C || !mode || (field != SMX_FIELD_B && field != SMX_FIELD_D)) return SMX_EINVAL;
    const HodgeHost& H = C->hodge[field == SMX_FIELD_B ? 0 : 1];
    *mode = H.separable ? 2 : H.mode;
    return SMX_OK;
}

int smx_cfl(smx_ctx* C, int iters, double tol, double* v, double* w, double* t, double* dt_max) {
    NEED_WS(C);
    if (!v || !w || !t || !dt_max || iters < 1 || !(tol >= 0.0)) return SMX_EINVAL;
    std::vector<double> v0(C->N_e);
    uint64_t state = 0x5eed5eedULL;
    for (auto& x : v0) x = (double)(splitmix64(state) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    CK(cudaMemcpyAsync(v, v0.data(), v0.size() * sizeof(double), cudaMemcpyHostToDevice, C->stream));
    double lam = 0.0, lam_old = 0.0;
    for (int it = 0; it < iters; ++it) {
        int st = hodge_apply_impl(C, 1, v, C->scratch);  // S = M~ v
        if (st) return st;
        if ((st = dot_impl(C, v, C->scratch, C->N_e, 0))) return st;  // den = v.M~v
        if ((st = solve_impl(C, 0, C->scratch, w))) return st;        // w = K_1^{-1} M~ v
        CK(cudaMemsetAsync(t, 0, C->N_h * sizeof(double), C->stream));
        if ((st = curl_primal_impl(C, w, t, 1.0))) return st;        // t = D^1 w
        if ((st = hodge_apply_impl(C, 0, t, C->scratch))) return st;  // S = M t
        if ((st = solve_impl(C, 1, C->scratch, t))) return st;        // t = K~_1^{-1} M t
        CK(cudaMemsetAsync(w, 0, C->N_e * sizeof(double), C->stream));
        if ((st = curl_dual_impl(C, t, w, 1.0, nullptr, nullptr, 0, 0.0))) return st;  // w = D~^1 t = T v
        if ((st = hodge_apply_impl(C, 1, w, C->scratch))) return st;  // S = M~ w
        if ((st = dot_impl(C, v, C->scratch, C->N_e, 1))) return st;  // num = v.M~ T v
        if ((st = dot_impl(C, w, C->scratch, C->N_e, 2))) return st;  // |T v|^2_M~
        double host[3];
        CK(cudaMemcpyAsync(host, C->dots, 3 * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
        CK(cudaStreamSynchronize(C->stream));
        if (!std::isfinite(host[0]) || !std::isfinite(host[1]) || !(host[2] > 0.0)) return SMX_ENONFINITE;
        lam = host[1] / host[0];
        const double sc = 1.0 / std::sqrt(host[2]);
        if ((st = run(C, 7, 1, [&] { return launch_scale_copy(w, v, sc, C->N_e, C->stream); }))) return st;
        if (it > 0 && std::fabs(lam - lam_old) <= tol * std::fabs(lam)) break;
        lam_old = lam;
    }
    if (!(lam > 0.0)) return SMX_ENONFINITE;
    *dt_max = 2.0 / std::sqrt(lam);
    return SMX_OK;
}

}  // extern "C"
