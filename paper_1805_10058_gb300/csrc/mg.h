// Multigrid (Section 6.1): Galerkin hierarchy with the block prolongator I_d (x) P (x) ... (x) P
// (eq:2by2prol), R = P^T, A_{l+1} = P^T A_l P (kept in Kronecker form through the coarse 1D
// bands), Chebyshev-Jacobi smoothing, dense per-solve inverse on the coarsest level.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "cd_internal.h"

namespace cd {

struct MgLevelBuf {
  void* b = nullptr;  // right-hand side of the level (levels >= 1)
  void* x = nullptr;  // iterate of the level (levels >= 1)
  void* r = nullptr;  // residual
  void* dv = nullptr;  // Chebyshev direction
  void* dinv = nullptr;  // 1 / diag(A_l) per solve, [B][N_l] (set by mg_prepare)
  void* xb = nullptr;    // second iterate buffer of the fused smoother (ping-pong)
};

struct MgData {
  int d = 0, P = 0, L = 0, B = 0, deg = 2;
  std::vector<int> ml;
  std::vector<long long> Nl;
  std::vector<size_t> boff;
  const double* bands64 = nullptr;
  const float* bands32 = nullptr;
  std::vector<Band> hM, hA, hS;
  std::vector<MgLevelBuf> lv64, lv32;
  std::vector<void*> owned;
  double* lmax = nullptr;     // [L][B] largest eigenvalue estimate of D^{-1} A_l
  double* cinv64 = nullptr;   // [B][nc][nc] coarsest inverse
  float* cinv32 = nullptr;
  int nc = 0;
  void* scratch64 = nullptr;  // 3D apply scratch of the finest level size
  void* scratch32 = nullptr;
  double* part = nullptr;     // partial sums [B][1024]
  double* tmpB = nullptr;     // [B]
  double* gjws = nullptr;     // side buffer of the coarsest inversion (nc >= 128)
  double alpha_cache_ok = 0;
  // Krylov post-smoother of the finest level (Section 6.1), set up by mg_setup_ksmooth:
  // ks_steps iterations; vectors (2 ks_steps + 2 of [B][N_0] per precision), per-solve scalars
  int ks_steps = 0;
  void* ks64 = nullptr;
  void* ks32 = nullptr;
  double *ks_H = nullptr, *ks_hc = nullptr, *ks_inv = nullptr, *ks_beta0 = nullptr, *ks_y = nullptr;
  double *ks_part = nullptr, *ks_rz = nullptr, *ks_a = nullptr, *ks_b = nullptr;
  const void *tLb64 = nullptr, *tLb32 = nullptr, *tdinv64 = nullptr, *tdinv32 = nullptr;  // T factor
  // second and later V-cycles of one preconditioner application: residual and correction
  void *cyc64 = nullptr, *cyc32 = nullptr;
  // hierarchy of the block diagonal D of eq:diag (P_WL): coupling blocks scaled by zero
  bool diag_only = false;
  double* gsc_zero = nullptr;
  ~MgData();
};

cd_status mg_build(MgData& mg, int d, int P, const std::vector<int>& ml,
                   const std::vector<Band>& hM, const std::vector<Band>& hA,
                   const std::vector<Band>& hS, int B, int deg, const double* bands64,
                   const float* bands32, const std::vector<size_t>& boff);
cd_status mg_set_params_slots(MgData& mg, int d, int P, const std::vector<double>& alpha,
                              const std::vector<double>& beta, const std::vector<int>& slots,
                              cudaStream_t s);
cd_status mg_set_params(MgData& mg, int d, int P, int nrhs, const std::vector<double>& alpha,
                        const std::vector<double>& beta, cudaStream_t s);

// Computes the Chebyshev bounds (power iteration on D^{-1} A_l, FP64) for the current
// per-solve parameters; must follow mg_set_params and the upload of alpha / beta.
cd_status mg_prepare(MgData& mg, int B, Coef c, double* fine_scratch64, cudaStream_t s);
// Finest-level post-smoothing of a V-cycle: Chebyshev (the parallel smoother of every level),
// or `steps` iterations of PGMRES / PCG preconditioned by T (Section 6.1, Section 6.2).
enum { kPostCheb = 0, kPostPgmres = 1, kPostPcg = 2 };
// Allocates the Krylov smoother's vectors and scalars (once) and records the banded factor of T
// (Lb, dinv in FP64 and FP32, as for launch_tband).
cd_status mg_setup_ksmooth(MgData& mg, int steps, const void* Lb64, const void* dinv64,
                           const void* Lb32, const void* dinv32);
// Turns the hierarchy into that of D = blockdiag(A^(c,c)) (eq:diag): every operator apply of the
// multigrid runs with the coupling blocks scaled by zero; call before mg_set_params.
cd_status mg_set_block_diagonal(MgData& mg);
// z = `cycles` V-cycles on A z = r from z = 0 (each later cycle corrects with the residual of
// the previous one); `post` selects the finest level's post-smoother.
template <typename T>
void mg_vcycle(MgData& mg, int d, int P, int B, const T* r, T* z, Coef c, const int* active,
               cudaStream_t s, T* fine_scr, int post = kPostCheb, int cycles = 1);
// the Krylov smoothers themselves (ksmooth.cu): xout = xin + ks_steps iterations on A x = b
template <typename T>
void ks_pgmres(MgData& mg, int B, const T* b, const T* xin, T* xout, Coef c, const int* active,
               T* scr, cudaStream_t s);
template <typename T>
void ks_pcg(MgData& mg, int B, const T* b, const T* xin, T* xout, Coef c, const int* active,
            T* scr, cudaStream_t s);
template <typename T>
void mg_restrict(int d, int mf, int mc, int B, const T* fine, T* coarse, const int* active,
                 cudaStream_t s);
template <typename T>
void mg_prolong_add(int d, int mf, int mc, int B, const T* coarse, T* fine, const int* active,
                    cudaStream_t s);

// Dense FP64 matrix of the operator on one level (Kronecker form), row-major n x n, n = d m^d.
std::vector<double> dense_operator(int d, const Band& M, const Band& A, const Band& S,
                                   double alpha, double beta);

}  // namespace cd
