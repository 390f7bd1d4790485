// Device-visible argument blocks and kernel launchers of the leapfrog path.
// Shared by kernels.cu (device code) and api.cu (the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace smx {

constexpr int kLMax = 16;      // max local functions per tile and axis (tile <= 8 elements, p <= 6)
constexpr int kTileMax = 8;    // max elements per Hodge tile and axis
constexpr int kRMax = 8;       // max local functions per element and axis (p + 1 <= 7)
constexpr int kPMax = 6;       // largest supported degree
constexpr int kSolveLines = 32;  // lines per CTA in the pairing sweeps
constexpr int kDotBlocks = 304;  // CTAs of the first reduction stage (2 x 152 SMs)
constexpr int kCurlThreads = 256;  // curl: points of a component plane per CTA
constexpr int kCurlKz = 2;         // curl: planes along z per thread (more CTAs: latency-bound stencil)

// One component of a field: extents (x, y, z) and offset in the global vector.
struct DevComp {
    int n[3];
    long long off;
};
struct DevField {
    DevComp c[3];
    long long total;
};

// Banded LU of one 1D factor (see BandLU in setup.h); device pointers.
struct DevFactor {
    const double* L;
    const double* U;
    const double* dinv;
    int n;
};

// Per-axis sweep of a pairing solve: for each component the factor along `axis`.
struct SolveArgs {
    DevField field;
    DevFactor f[3];
    int axis;
};

// Fused line pass of a separable Hodge star: x = A^{-1} (M y) along one axis,
// M the univariate mass of the component's space along that axis (banded,
// half-bandwidth = the space's degree), A the pairing factor.
struct MassSolveArgs {
    DevField field;
    DevFactor f[3];
    const double* mass[3];   // per component: n x (2 deg + 1) band rows, zero padded
    int deg[3];              // per component: mass half-bandwidth
    int axis;
};

// Block-Kronecker Hodge apply: M = sum_t gamma_t (Mz_t (x) My_t (x) Mx_t).
struct HodgeBlockArgs {
    DevField field;
    int ntile[3];
    int kinds[3][3];   // kinds[c][a]
    int deg[3][3];     // degree of kinds[c][a]
    const int* tf0[3];       // tf0[a][kind * ntile[a] + t]: first local function of tile t
    const int* tlen[3];      // number of local functions
    const double* tmat[3];   // (kind * ntile[a] + t) * kLMax^2: dense tile mass, row-major
    const double* gamma;     // per tile, x fastest
    int max_nloc;            // largest Lx*Ly*Lz over tiles and components (sizes shared memory)
};

// Quadrature Hodge apply (curved map or pointwise material).
struct HodgeQuadArgs {
    DevField field;
    int nel[3];
    int q[3];
    int kinds[3][3];
    int deg[3][3];
    int koff[3][3];          // index shift of kinds[c][a] (-1 for P0)
    const double* bval[3];   // ((kind * nel[a] + e) * q[a] + qp) * kRMax + r
    const double* G;         // 6 arrays of Qtot: G00 G01 G02 G11 G12 G22 (weight, metric, material folded in)
    long long Qtot;
    int Qn[3];               // quadrature points per axis
};

// ---- FP32 operators of the mixed-precision step (kernels_f32.cu): split (hi, lo) coefficients
struct HodgeBlockF32Args {
    DevField field;
    int ntile[3];
    int kinds[3][3];
    int deg[3][3];
    const int* tf0[3];
    const int* tlen[3];
    const float2* tmat[3];
    const double* gamma;
    int max_nloc;
    int max_len[2];      // largest tile length along x and y over the field's components (the CTA shape)
    int compensated;     // nonzero: compensated FP32 sums of products in the tile passes (refined form)
};

// FP32 quadrature Hodge apply: HodgeQuadArgs with FP32 basis values and metric.
struct HodgeQuadF32Args {
    DevField field;
    int nel[3];
    int q[3];
    int kinds[3][3];
    int deg[3][3];
    int koff[3][3];
    const float2* bval[3];   // (hi, lo) pairs
    const float2* G;         // (hi, lo) pairs, 6 arrays of Qtot
    long long Qtot;
    int Qn[3];
};

struct LineF32Args {
    DevField field;
    const float2* L[3];     // per component: n x KL
    const float2* U[3];     // per component: n x KL (divided by the diagonal)
    const float2* dinv[3];  // per component: n
    const float2* mass[3];  // per component: n x (2 deg + 1) band rows (fused separable star only)
    int deg[3];
    int axis;
};

// Dense mode product along one axis: every line x of component c becomes B[c] x.
struct ModeF32Args {
    DevField field;
    const float2* B[3];  // per component: B^T, n rows of npad (hi, lo) pairs (zero past n)
    int axis;
    int npad;            // mode_f32_npad(max line length)
};
constexpr int kModeMaxN = 80;  // largest line length the mode-product kernel handles

cudaError_t launch_mode_f32(const ModeF32Args& a, const double* in64, const float* in32, float* out, cudaStream_t s);
int mode_f32_npad(int maxn);  // padded output count of the CUDA-core kernel for lines up to maxn

// Mode products on the tensor cores by exact digit slicing (kernels_f64tc.cu):
// the operator's rows and the lines cut into balanced base-256 digits (BF16
// exact), digit levels accumulated exactly in FP32 tensor memory.
// Operator table (digit_split_operator, setup.h): per component, uint16 BF16
// patterns of the digit planes in the K-major 32-byte swizzle layout, plus the
// rows' exponent fields (int32, one per row).
constexpr int kDigits = 7;     // FP64 step: 55-bit fixed point, levels 0..6
constexpr int kDigitsF32 = 4;  // mixed step: 31-bit fixed point, levels 0..3
struct ModeDigitArgs {
    DevField field;
    const void* B[3];       // per component: digit planes of the operator
    const int* rowexp[3];   // per component: largest exponent field of each operator row (>= 1)
    int npad[3];            // per component: line length rounded up to a multiple of 16
    int axis;
    unsigned* status;       // device word: bit 0 set when an MMA completion wait gave up
};
int mode_digit_npad(int n);
// out = B in along the axis, FP64 in and out (in == out allowed: each tile reads before it writes);
// the operator table of kDigits planes.
cudaError_t launch_mode_digit(const ModeDigitArgs& a, const double* in, double* out, cudaStream_t s);
// The mixed step's version with kDigitsF32 planes: input FP64 (in64) or FP32 (in32), output FP32,
// and optionally the result also widened to FP64 (out64).
cudaError_t launch_mode_digit_f32(const ModeDigitArgs& a, const double* in64, const float* in32, float* out,
                                  double* out64, cudaStream_t s);
// zero (optional): also set zero[i] = 0 for every output index i (the accumulation
// target of the Hodge apply that follows the curl).
cudaError_t launch_curl_f32(bool dual, const DevField& IN, const DevField& OUT, const float* in, double* out,
                            double alpha, const double* jhat, const double* amp, int amp_index, double s_host,
                            cudaStream_t s, double* zero = nullptr);
// Banded 1D pairing factor applied along one axis (the FP64 residual of the
// refined mixed step): out = A x along every line of the axis, or out = y - A x
// when y is given.  x is FP64 (in64) or FP32 (in32); A in band rows.
struct BandApplyArgs {
    DevField field;
    const double* band[3];  // per component: n x (2 kl + 1) band rows, row m holds A(m, m - kl .. m + kl)
    int kl;                 // half-bandwidth (degree along the axis - 1)
    int axis;
};
cudaError_t launch_band_apply(const BandApplyArgs& a, const double* in64, const float* in32, const double* y,
                              double* out, cudaStream_t s);
// out = x0 + c in FP64 (both FP32; the sum is exact in FP64 unless the exponents differ by more than 29)
cudaError_t launch_refine_sum(const float* x0, const float* c, double* out, long long n, cudaStream_t s);
cudaError_t launch_cast_d2f(const double* x, float* y, long long n, cudaStream_t s);
cudaError_t launch_cast_f2d(const float* x, double* y, long long n, cudaStream_t s);
cudaError_t launch_hodge_block_f32(const HodgeBlockF32Args& a, const double* x64, const float* x32, double* y,
                                   cudaStream_t s);
cudaError_t launch_hodge_quad_f32(const HodgeQuadF32Args& a, const double* x, double* y, cudaStream_t s);
cudaError_t launch_line_f32(const LineF32Args& a, int kl, bool mass, const double* in64, const float* in32, float* out,
                            cudaStream_t s);

// ---- reverse step and receivers (kernels_adj.cu)
// Receiver rows in CSR form: row r = 3 * point + component of the E field.
struct RecArgs {
    const int* ptr;      // nrows + 1
    const int* idx;      // entry -> index into e
    const double* val;   // entry -> basis value
    int nrows;
};
// Per-block derivative of the electric mass: block layout and scale[c] = -1/eps_c.
struct PairArgs {
    const double* scale;     // per block
    const int* tile_block;   // block-Kronecker Hodge: block of each tile
    int epb[3];              // elements per block along x, y, z
    int nb[3];               // blocks along x, y, z
};
cudaError_t launch_receivers_eval(const RecArgs& r, const double* e, double* out, cudaStream_t s);
cudaError_t launch_receivers_adjoint(const RecArgs& r, const double* w, double alpha, double* ebar, cudaStream_t s);
cudaError_t launch_axpy(const double* x, double* y, double a, long long n, cudaStream_t s);
cudaError_t launch_rescale_metric(double* G64, float2* G32, const HodgeQuadArgs& a, const int epb[3], const int nb[3],
                                  const double* ratio, cudaStream_t s);
cudaError_t launch_hodge_quad_pair(const HodgeQuadArgs& a, const PairArgs& p, const double* z, const double* d,
                                   double* out, cudaStream_t s);
cudaError_t launch_hodge_block_pair(const HodgeBlockArgs& a, const PairArgs& p, const double* z, const double* x,
                                    double* out, cudaStream_t s);

// ---- batched cavities: one persistent launch per leapfrog step (kernels.cu)
// FP64 cavities of any map and material: each Hodge star is either the fused mass + solve passes
// (identity map, constant material: sep) or a mass apply (block-Kronecker tiles on the identity
// map, quadrature elements otherwise) into the cavity's scratch vector y followed by the pairing
// sweeps.  Per cavity: its field layouts, the argument blocks of its own context, state, scratch.
struct BatchCavity {
    DevField fE, fB, fH, fD;
    MassSolveArgs msH[3];     // star of B, sepB: fused mass + K~_1 solve per axis
    MassSolveArgs msD[3];     // star of D, sepD
    SolveArgs solveH[3];      // K~_1 sweeps (star of B otherwise)
    SolveArgs solveE[3];      // K_1 sweeps (star of D otherwise)
    HodgeBlockArgs hbB, hbD;  // block-Kronecker mass applies (mode 0)
    HodgeQuadArgs hqB, hqD;   // quadrature mass applies (mode 1)
    double *d, *b, *e, *h, *y;
    const double* jhat;       // or null
    const double* amp;        // device, one value per step (with jhat)
    double dt;
    int kl[3];                // p - 1 per axis
    int sepB, sepD;           // fused star
    int modeB, modeD;         // mass apply otherwise: 0 block tiles, 1 quadrature elements
};
constexpr int kBatchPhases = 11;
constexpr int kBatchThreads = 256;
struct BatchArgs {
    const BatchCavity* cav;
    const int2* items[kBatchPhases];   // per phase: (cavity, unit)
    int nitems[kBatchPhases];
    unsigned* bar;          // [0] arrivals, [1] generation
    unsigned* status;       // bit 1: a grid barrier gave up
    int line_warps;         // warps of a CTA that take line items
    int warp_smem;          // doubles of shared memory per line warp
    int step;               // index into amp (when stepctr is null)
    unsigned* stepctr;      // device step counter: read at entry, advanced by CTA 0 at the end (graph replays)
    unsigned long long wait_ns;  // limit of each grid-barrier wait (default one second)
};
// unit encodings
__host__ __device__ inline int batch_curl_unit(int c, int pb, int zc) { return (c << 28) | (zc << 14) | pb; }
__host__ __device__ inline int batch_zero_unit(int z) { return (1 << 30) | z; }
__host__ __device__ inline int batch_comp_unit(int c, int k) { return (c << 24) | k; }
size_t hodge_quad_smem_doubles(int qx, int qy, int qz);
cudaError_t launch_batch_step(const BatchArgs& a, int grid, size_t smem, cudaStream_t s);
int batch_blocks_per_sm(size_t smem);
size_t batch_line_warp_doubles(int maxn, int kl);  // staging of one line warp

// The refined mixed step (FP32 operators, one FP64-residual refinement per Kronecker solve,
// FP64 state and star outputs) of many cavities in one persistent launch (kernels_f32.cu):
// twenty-five phases separated by grid barriers,
//   0 b -= dt/2 D^1 e; y = 0      1 y = M b (FP32 products, FP64 sums)
//   2-4 x0 = K~_1^{-1} y per axis (FP32 line sweeps)
//   5-7 t = y - K~_1 x0 (FP64 band applies per axis)
//   8-10 c = K~_1^{-1} t per axis 11 h = x0 + c
//   12 d += dt (D~^1 h - s jhat); y = 0   13-23 the same for the star of D (e)
//   24 b -= dt/2 D^1 e
constexpr int kRefPhases = 25;
struct BatchRefCavity {
    DevField fE, fB, fH, fD;
    DevField fS[2];             // layout of each star's mass apply and solves (B, D)
    HodgeBlockF32Args hb[2];    // [0] star of B (M^2), [1] star of D (M~^2)
    HodgeQuadF32Args hq[2];
    int mode[2];                // mass apply: 0 block tiles, 1 quadrature elements
    LineF32Args ln[2][3];       // FP32 pairing sweeps per star and axis
    BandApplyArgs band[2][3];   // FP64 band rows of the pairing factors per star and axis
    int kl[3];                  // p - 1 per axis
    double *d, *b, *e, *h;      // state
    double *y, *t64, *s64;      // mass apply, residual, residual scratch (FP64)
    float* x0[2];               // first FP32 solution of each star
    float* c32;                 // FP32 correction
    const double* jhat;         // or null
    const double* amp;          // device, one value per step (with jhat)
    double dt;
};
struct BatchRefArgs {
    const BatchRefCavity* cav;
    const int2* items[kRefPhases];
    int nitems[kRefPhases];
    unsigned* bar;
    unsigned* status;
    int line_warps;
    int warp_floats;            // floats of shared memory per line warp
    int step;
    unsigned* stepctr;
    unsigned long long wait_ns;
};
cudaError_t launch_batch_refined_step(const BatchRefArgs& a, int grid, size_t smem, cudaStream_t s);
int batch_refined_blocks_per_sm(size_t smem);
size_t batch_ref_line_warp_floats(int maxn, int kl);           // staging of one FP32 line warp
size_t batch_ref_mass_floats(int max_nloc, int qx, int qy, int qz);  // largest FP32 mass unit (q = 0: none)

// ---- launchers (kernels.cu); all enqueue on `s` and return cudaGetLastError()
cudaError_t launch_curl_primal(const DevField& E, const DevField& B, const double* e, double* b,
                               double alpha, cudaStream_t s, double* zero = nullptr);
cudaError_t launch_curl_dual(const DevField& H, const DevField& D, const double* h, double* d,
                             double alpha, const double* jhat, const double* amp, int amp_index,
                             double s_host, cudaStream_t s, double* zero = nullptr);
cudaError_t launch_hodge_block(const HodgeBlockArgs& a, const double* x, double* y, cudaStream_t s);
cudaError_t launch_hodge_quad(const HodgeQuadArgs& a, const double* x, double* y, cudaStream_t s);
cudaError_t launch_solve_axis(const SolveArgs& a, int kl, const double* in, double* out, cudaStream_t s);
cudaError_t launch_mass_solve_axis(const MassSolveArgs& a, int kl, const double* in, double* out, cudaStream_t s);
// partial[b] of sum_i x_i y_i over kDotBlocks CTAs, then out[0] = total (device)
cudaError_t launch_dot(const double* x, const double* y, long long n, double* partial, double* out,
                       cudaStream_t s);
cudaError_t launch_scale_copy(const double* x, double* y, double a, long long n, cudaStream_t s);
cudaError_t launch_zero(double* y, long long n, cudaStream_t s);  // y = 0 as a kernel of the launch chain

// ---- preconditioned conjugate gradients of scheme 1 (kernels.cu); scalars live on the device:
// scal[0] = r.z, scal[1] = p.Ap, scal[2] = r.r, scal[3] = new r.z, scal[4] = y.y
enum CgScalar { kCgRz = 0, kCgPAp = 1, kCgRr = 2, kCgRzNew = 3, kCgYy = 4, kCgCount = 5 };
// x += alpha p, r -= alpha Ap with alpha = r.z / p.Ap (0 when p.Ap = 0)
cudaError_t launch_cg_xr(double* x, double* r, const double* p, const double* Ap, const double* scal, long long n,
                         cudaStream_t s);
// p = z + beta p with beta = new r.z / r.z (0 when r.z = 0); then r.z = new r.z (one thread, after the grid:
// a second tiny kernel)
cudaError_t launch_cg_p(double* p, const double* z, double* scal, long long n, cudaStream_t s);
// r = y - r (in place: r holds M x on entry)
cudaError_t launch_sub_from(const double* y, double* r, long long n, cudaStream_t s);
cudaError_t launch_copy(const double* x, double* y, long long n, cudaStream_t s);

}  // namespace smx
