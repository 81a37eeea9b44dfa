// Internal declarations shared by the host setup code, the kernels and the solver.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/curldiv.h"

namespace cd {

// ------------------------------------------------------------------ error handling
void set_error(const std::string& msg);
const char* last_error();
void count_launch(int k = 1);

#define CD_CUDA_OK(expr)                                                    \
  do {                                                                      \
    cudaError_t e_ = (expr);                                                \
    if (e_ != cudaSuccess) {                                                \
      ::cd::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));  \
      return CD_ECUDA;                                                      \
    }                                                                       \
  } while (0)

// ------------------------------------------------------------------ host setup
// 1D banded matrix: rows 0..m-1, row i holds entries (i, i-P .. i+P).
struct Band {
  int m = 0, P = 0;
  std::vector<double> v;  // m * (2P+1)
  double at(int i, int j) const {
    int k = j - i + P;
    return (k < 0 || k > 2 * P || j < 0 || j >= m) ? 0.0 : v[(size_t)i * (2 * P + 1) + k];
  }
};

// B-spline mass / advection / stiffness bands of degree p on n intervals,
// restricted to the Dirichlet basis N_2..N_{n+p-1} (m = n+p-2), half-band P >= p.
void iga_bands(int p, int n, int P, Band& M, Band& A, Band& S);
// T_m(m_{p-1}): entries phi_{2p-1}(p - i + j), |i-j| < p.
void toeplitz_T_band(int p, int m, int P, Band& T);
// Galerkin coarsening of a 1D band with the 3-tap prolongator (1/2, 1, 1/2).
Band coarsen(const Band& X);
// Dense symmetric (generalized) eigen-decompositions, FP64: Householder tridiagonalisation and
// implicit shifted QR (generalized: Cholesky reduction of M first).
// gen = true: solve S U = M U lam with U^T M U = I (M SPD); else T U = U lam.
bool sym_eig(int m, const std::vector<double>& Adense, std::vector<double>& U,
             std::vector<double>& lam);
bool gen_eig(int m, const std::vector<double>& Mdense, const std::vector<double>& Sdense,
             std::vector<double>& U, std::vector<double>& lam);
std::vector<double> band_to_dense(const Band& X);
// Banded Cholesky T_m(m_{p-1}) = L L^T, half-bandwidth q = p - 1: Lb[i * q + t] = L(i, i-q+t)
// for t < q ((m + q) x q, zero where the column is < 0 and in the q rows past m),
// dinv[i] = 1 / L(i, i).  False if a pivot is not positive.
bool tband_factor(int p, int m, std::vector<double>& Lb, std::vector<double>& dinv);
// Cholesky inverse of a small dense SPD matrix (FP64); false if not SPD.
bool spd_inverse(int n, std::vector<double>& a);

// ------------------------------------------------------------------ kernel launchers
struct Coef {  // per-solve operator coefficients, device arrays of length >= B
  const double* alpha;
  const double* beta;
  // scale of the coupling blocks gamma = alpha - beta (NULL: 1 for every solve).  0 gives the
  // block diagonal D = blockdiag(A^(c,c)) of eq:diag with the same kernels.
  const double* gsc = nullptr;
};

// Chebyshev smoother interval on D^{-1} A: [kChebHi lambda_max / kChebRatio, kChebHi lambda_max]
constexpr double kChebHi = 1.1, kChebRatio = 30.0;

// Epilogue of mode 2 (a Chebyshev smoothing step fused into the apply): with r = rhs - A w at
// each output point and 1/diag(A) computed from the 1D band diagonals,
//   d = (step == 0) ? r / (theta diag) : c1 dprev + c2 r / diag,   xout = xprev + d,
// optionally dout = d and rout = r.  Nothing is written to y.  (dprev, xprev are read only at
// the output point; w is read with halos, so w must not alias xout, dout or rout.)
template <typename T>
struct Epi {
  const T* dprev;
  const T* xprev;
  T* xout;
  T* dout;
  T* rout;
  const double* lmax;  // per solve: largest eigenvalue estimate of D^{-1} A
  int step;
  const T* dinv = nullptr;  // 1 / diag(A) per solve ([B][N]); kernels that do not read it
                            // form the diagonal from the 1D band diagonals
};

// y = A w (mode 0) or y = b - A w (mode 1) on one level; optional per-solve partial dots
// dotp[b * nblk + blk] = sum over the block of w * y (mode 0) or y * y (mode 1).
template <typename T>
int launch_apply(int d, int m, int P, const T* bands /*M,A,S*/, const T* w, T* y,
                 const T* rhs, int mode, int B, Coef c, double* dotp, int* nblk,
                 const int* active, T* scratch, cudaStream_t s, const Epi<T>* epi = nullptr);

// y = A w (mode 0) or rhs - A w (mode 1) on an anisotropic mesh: ma[l] unknowns per component
// along x_l, band[l] the [3][ma[l]][2P+1] row-major (M, A, S) bands of direction l; scratch holds
// 6 (d = 2) or 18 (d = 3) arrays of [B][prod ma] plus a [B][N] buffer.
template <typename T>
int launch_apply_aniso(int d, const int* ma, int P, const T* const* band, const T* w, T* y,
                       const T* rhs, int mode, int B, Coef c, double* dotp, int* nblk,
                       const int* active, T* scratch, cudaStream_t s);
// FD-D scaling on an anisotropic mesh: z /= sum_l c_{comp,l} lam_l[k_l] (eigen-coordinates)
template <typename T>
void launch_fd_scale_aniso(int d, const int* ma, const T* const* lam, int B, const double* alpha,
                           const double* beta, T* z, const int* active, cudaStream_t s);

// Serving sessions on a handle (iteration-level continuous batching; the handle's max_batch
// slots; a handle in session use must not run batched calls meanwhile).
int sess_busy(cd_solver h);
cd_status sess_admit(cd_solver h, const double* b_host, double alpha, double beta, int* slot);
cd_status sess_step(cd_solver h, std::vector<int>& finished);
cd_status sess_take(cd_solver h, int slot, double* x_host, cd_result* res);

// Central-stencil registry for the 2D apply: `bands_dev` is the start of a level's band
// block ([3][m][W] row-major, then [3][W][m] k-major); rows [lo, hi) equal `central`
// ([3][W]: M, A, S).
void register_level(const void* bands_dev, int m, int P, int lo, int hi, const double* central);
void unregister_level(const void* bands_dev);
// FP64 levels: also a (hi, lo) FP32 split of the k-major bands, for the double-FP32 apply.
void register_level_ff(const double* bands_dev, int m, int P);
// 2D apply kernel: 2 = v3 (x_2 first, packed pairs; default), 1 = v2, 0 = v1.
void set_apply_variant(int v);
// 3D apply: 1 = streaming fused kernel (default), 0 = three banded passes (kept for checks).
void set_apply3d_variant(int v);
void set_apply_fp64_variant(int v);  // 2D FP64: 0 = v2, 1 = v3, 2 = double-FP32 everywhere
// double-FP32 2D apply tile rows: 0 = chosen by the grid size, 8 = narrow tile, else wide tile
void set_ff2_rows(int rows);
int num_sms();  // SMs of the current device (cached after the first call)
// The calling thread's FP64 2D applies (modes 0 and 1) run in double-FP32 arithmetic on the
// FP32 pipe while set (the inner FP64 Krylov solves of the refinement loop); fp64_emulated()
// tells whether they do now.
void set_fp64_emulated(int on);
int fp64_emulated();

// Autotuner of the 2D apply: times the variants on (m, P, B) and records the fastest
// (returns the chosen variant, 0 if none was tuned).  Not inside a stream capture.
template <typename T>
int tune_apply2d(int m, int P, const T* bands, const T* w, T* y, int B, Coef c, cudaStream_t s);

// Autotuner of the 3D apply: times the streaming kernel against the three banded passes on
// (m, P, B) and records the faster (returns 1 streaming, 2 passes).  Not inside a stream capture.
template <typename T>
int tune_apply3d(int m, int P, const T* bands, const T* w, T* y, int B, Coef c, T* scratch,
                 cudaStream_t s);

template <typename T>
bool apply_can_fuse(int d, int m, int P, const T* bands, int B);

// Sets kernel attributes (dynamic shared memory caps); call once before launches/captures.
int prepare_kernels();

// Extended-precision outer residual (ext_residual.cu): r = b - A (xh + xl) in double-FP64 from
// the FP64 bands of the finest level, rounded to FP64 (xl may be NULL).  `scratch` holds
// chunk * ext_scratch_doubles_per_solve(d, m) doubles; solves are processed `chunk` at a time.
long long ext_scratch_doubles_per_solve(int d, int m);
int launch_ext_residual(int d, int m, int P, const double* bands, const double* rhs,
                        const double* xh, const double* xl, double* r, int B, Coef c,
                        const int* active, double* scratch, int chunk, cudaStream_t s);
// (xh, xl) += rnorm_b * e, exactly rounded into the double-FP64 pair
template <typename E>
void launch_ext_update(long long N, int B, double* xh, double* xl, const E* e,
                       const double* rnorm, const int* active, cudaStream_t s);

// capacity (per solve) of the block-partial-sum arrays every reduction writes into
constexpr int kMaxPartials = 4096;

// generic reductions / vector kernels (per solve, deterministic)
int partial_blocks(long long N);
template <typename T>
int launch_dot(const T* a, const T* b, long long N, int B, double* part, int nblk,
               const int* active, cudaStream_t s);
int launch_sum_partials(const double* part, int nblk, int B, double* out, cudaStream_t s);

}  // namespace cd
