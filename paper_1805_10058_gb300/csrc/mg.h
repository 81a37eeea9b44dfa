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
  double alpha_cache_ok = 0;
  ~MgData();
};

cd_status mg_build(MgData& mg, int d, int P, const std::vector<int>& ml,
                   const std::vector<Band>& hM, const std::vector<Band>& hA,
                   const std::vector<Band>& hS, int B, int deg, const double* bands64,
                   const float* bands32, const std::vector<size_t>& boff);
cd_status mg_set_params(MgData& mg, int d, int P, int nrhs, const std::vector<double>& alpha,
                        const std::vector<double>& beta, cudaStream_t s);

// Computes the Chebyshev bounds (power iteration on D^{-1} A_l, FP64) for the current
// per-solve parameters; must follow mg_set_params and the upload of alpha / beta.
cd_status mg_prepare(MgData& mg, int B, Coef c, double* fine_scratch64, cudaStream_t s);
// z = one V-cycle applied to r, from a zero initial guess.
template <typename T>
void mg_vcycle(MgData& mg, int d, int P, int B, const T* r, T* z, Coef c, const int* active,
               cudaStream_t s, T* fine_scr);
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
