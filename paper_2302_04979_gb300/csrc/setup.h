// Host-side FP64 setup of the spline geometric leapfrog (not timed).
//
// Univariate spaces (Sec. 2.3 and the basis choice of Sec. 4.1): on each axis
// with degree p and nel uniform elements, n = nel + p,
//   kind P0: primal S_p(Xi) B-splines, first and last removed (BC)   dim n-2
//   kind P1: primal S_{p-1}(Xi') Curry-Schoenberg                     dim n-1
//   kind D0: dual   S_{p-1}(Xi') B-splines                            dim n-1
//   kind D1: dual   S_{p-2}(Xi'') Curry-Schoenberg                    dim n-2
// On element e every kind of degree d has the d+1 functions e..e+d of its
// full (open-knot) basis; P0 shifts that index by -1 and drops 0 and n-1.
#pragma once

#include <cstdint>
#include <vector>

namespace smx {

enum Kind { P0 = 0, P1 = 1, D0 = 2, D1 = 3 };

// Space kinds along (x, y, z) of component c of each field (E, B, H, D).
extern const int kFieldKinds[4][3][3];

int kind_degree(int kind, int p);
int kind_dim(int kind, int p, int nel);
// index shift from the full basis numbering to the stored numbering (-1 for P0)
int kind_offset(int kind);

// Gauss-Legendre rule on [0,1] by Newton iteration on the Legendre recurrence.
void gauss_legendre01(int q, std::vector<double>& x, std::vector<double>& w);

// Values of the d+1 basis functions of one kind that live on element e, at a
// point x inside that element (full-basis numbering e..e+d; CS scaling applied).
void local_basis(int kind, int p, int nel, int e, double x, double* out);

// Dense univariate pairing matrix int phi_i psi_j (row kind, column kind), row-major.
std::vector<double> pairing_matrix(int row_kind, int col_kind, int p, int nel);

// Banded LU without pivoting: A = L U, L unit lower with kl sub-diagonals, U
// upper with ku super-diagonals.  Returns false on a pivot below
// tol * max|A| (the factor is then unusable).
struct BandLU {
    int n = 0, kl = 0, ku = 0;
    std::vector<double> L;     // L[i*kl + k-1] = L(i, i-k), k = 1..kl
    std::vector<double> U;     // U[i*ku + k-1] = U(i, i+k) / U(i,i), k = 1..ku
    std::vector<double> dinv;  // 1 / U(i,i)
};
bool band_lu(const std::vector<double>& A, int n, int kl, int ku, BandLU& out);
// Rebuild the dense matrix L * U (row-major) from a factor.
std::vector<double> band_lu_dense(const BandLU& f);

// Geometry map F (SMX_GEOM_IDENTITY, or SMX_GEOM_SINE_BUMP with amplitude a)
// and its Jacobian, J[3 i + j] = dF_i / dxhat_j, at a parametric point; det3 of J.
void geometry_eval(int geom, double a, const double xh[3], double X[3], double J[9]);
double det3(const double J[9]);

// A geometry map: one of the built-in maps (kind SMX_GEOM_IDENTITY, or
// SMX_GEOM_SINE_BUMP with amplitude amp) or a host callback (SMX_GEOM_CALLBACK)
// that fills x[3 i + r] = F_r and jac[9 i + 3 r + c] = dF_r / dxhat_c at the n
// parametric points xh[3 i + c].
typedef void (*geometry_fn)(int64_t n, const double* xh, double* x, double* jac, void* user);
struct GeomMap {
    int kind = 0;
    double amp = 0.0;
    geometry_fn fn = nullptr;
    void* user = nullptr;
};
// F and J_F at n points (one callback call for a callback map).  Returns SMX_OK, or
// SMX_EGEOM if a value is not finite or det J_F <= 0 at some point.
int geometry_eval_points(const GeomMap& g, int64_t n, const double* xh, double* X, double* J);

// L2 projection of a physical 2-form onto X~^2 (field SMX_FIELD_D) or X^2_{h,0}
// (SMX_FIELD_B) (project.cpp): fn(n, xyz, out) fills out[3 i + c] with the
// vector proxy at the physical points xyz[3 i ..]; out (host, the field's
// length) receives the coefficients.  Preconditioned CG to ||r|| <= rtol ||b||.
// Returns SMX_OK, SMX_ENONFINITE (fn gave a non-finite value) or
// SMX_ESINGULAR (no convergence in maxit iterations).
typedef void (*project_fn)(int64_t n, const double* xyz, double* out, void* user);
int l2_project_2form(const int p[3], const int nel[3], const GeomMap& geom, int field, project_fn fn, void* user,
                     double* out, double rtol, int maxit, int* iters);

// Element mass matrix of one kind on element e: (d+1) x (d+1), row-major,
// int_e phi_i phi_j with q = p+1 Gauss points.
std::vector<double> element_mass(int kind, int p, int nel, int e);


// Digit planes of a dense n x n row-major FP64 operator B for the tensor-core
// mode products with nd digits (7: FP64 step, 4: mixed step): every row i is
// scaled by a power of two from F_i, its largest exponent field (at least 1),
// rounded to an integer X with |X| < 2^(8 nd - 1) (the row's largest
// significand shifted left by 8 nd - 1 - 53) and written as nd balanced
// base-256 digits X = sum_s e_s 256^(nd-1-s), e_s in [-128, 127] (e_0 in
// [-128, 128]), integer arithmetic only.
// planes: BF16 patterns in the K-major 32-byte swizzle layout, digit s,
// element (row i, column k) at uint16 index
//   s * (npad / 16) * r8 * 16 + (k / 16) * r8 * 16 + 16 i + 8 (((k / 8) & 1) ^ ((i / 4) & 1)) + k % 8,
// r8 = n rounded up to 8, zero outside n x n.  rowexp: F_i for i < n.
void digit_split_operator(const std::vector<double>& B, int n, int npad, int nd, std::vector<uint16_t>& planes,
                          std::vector<int32_t>& rowexp);
// The digits of one value for a given F (d[0..nd-1], most significant first).
void digits_fixed(double v, int F, int nd, int* d);

}  // namespace smx
