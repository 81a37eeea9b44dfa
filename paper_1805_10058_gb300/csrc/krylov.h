// Declarations of the Krylov / FD launch wrappers (krylov.cu) and multigrid kernels (mg.cu).
#pragma once
#include "cd_internal.h"

namespace cd {

// Per-solve scalar state of a (flexible) preconditioned CG, device arrays of length B.
struct PcgState {
  double* rz;
  double* rr;
  double* rr0;
  double* alpha;
  double* beta;
  double* rzold;
  int* active;
  int* iters;
  int* status;
};

// Epilogue of the last forward FD pass: divide by sum_l c_{comp,l} lam[k_l] (mode 1, FD of
// the block diagonal D, c = beta on the component's own axis and alpha elsewhere) or by
// prod_l lam[k_l] (mode 2, FD of T).  `base` is the start of the output tensor.
template <typename T>
struct FdScale {
  int mode;
  int d, m;
  long long per;  // m^d
  const T* lam;
  const double* alpha;
  const double* beta;
  const T* base;
};

template <typename T>
int launch_fd_axis(int d, int m, int axis, int B, const T* G, const T* in, T* out,
                   FdScale<T> sc, const int* active, cudaStream_t s);
// the contraction along `axis` of an anisotropic tensor (ma[l] entries along x_l), no scaling
template <typename T>
int launch_fd_axis_aniso(int d, const int* ma, int axis, int B, const T* G, const T* in, T* out,
                         const int* active, cudaStream_t s);

// z = T^{-1} r with T = I_d (x) T_m (x) ... (eq:kron_precond) by banded Cholesky solves along
// every axis (the banded factorisation route of Section 6.1).  T_m = L L^T with L lower banded
// of half-bandwidth q = p - 1: Lb[i * q + t] = L(i, i - q + t) for t < q ((m + q) x q, rows
// past m and entries left of column 0 zero), dinv[i] = 1 / L(i, i).  in == out is allowed.
template <typename T>
int launch_tband(int d, int m, int q, int B, const T* Lb, const T* dinv, const T* in, T* out,
                 const int* active, cudaStream_t s);

// tcgen05 (TF32) version of launch_fd_axis<float>; fd_tc_error() reports a bounded wait that
// expired inside the kernel (then its output is not written).
bool launch_fd_axis_tc(int d, int m, int axis, int B, const float* G, const float* in, float* out,
                       FdScale<float> sc, cudaStream_t s);
int fd_tc_error();

template <typename T>
void vcopy(long long N, int B, const T* src, T* dst, const int* active, cudaStream_t s);
template <typename T>
void vzero(long long N, int B, T* dst, const int* active, cudaStream_t s);
template <typename T>
void cg_update(long long N, int B, int nblk, T* x, T* r, const T* p, const T* q, const T* zold,
               const double* alpha, const int* active, double* part_rr, double* part_rz,
               cudaStream_t s);
template <typename T>
void xpay(long long N, int B, const T* z, T* p, const double* beta, const int* active,
          cudaStream_t s);
void ir_cast(long long N, int B, const double* r64, float* r32, const double* rnorm,
             const int* active, cudaStream_t s);
void ir_update(long long N, int B, double* x64, const float* e32, const double* rnorm,
               const int* active, cudaStream_t s);
// starts PCG for the solves in outer_active; the others are stopped (active = 0), or left as
// they are with keep_others (a session's solves that are mid-way through their own PCG)
void cg_init(int B, PcgState st, const double* prr, int nrr, const double* prz, int nrz,
             const int* outer_active, cudaStream_t s, int keep_others = 0);
void cg_alpha(int B, PcgState st, const double* ppq, int npq, cudaStream_t s);
void cg_check(int B, PcgState st, const double* prr, int nrr, const double* prz, int nrz,
              const double* tol2v, int maxit, cudaStream_t s);
void cg_beta(int B, PcgState st, const double* prz, int nrz, int flexible, cudaStream_t s);
void count_active(int B, const int* active, int* out, cudaStream_t s);
void ir_check(int B, const double* prr, int nrr, const double* bnorm2, double* rnorm,
              double* rrprev, int* active, int* status, double* relres, int* outer_it, int* grp,
              double* tol2v, double tol2, double inner2, int max_outer, const int* inner_total,
              int maxit, double floor2, cudaStream_t s);
void group_masks(int B, const int* active, const int* grp, int* m0, int* m1, int* m2, int* out,
                 cudaStream_t s);
void scale_div(long long N, int B, const double* src, double* dst, const double* rnorm,
               const int* active, cudaStream_t s);
void ir_update64(long long N, int B, double* x64, const double* e, const double* rnorm,
                 const int* active, cudaStream_t s);
void to_f32(long long N, int B, const double* src, float* dst, const int* active, cudaStream_t s);
void to_f64(long long N, int B, const float* src, double* dst, const int* active, cudaStream_t s);

}  // namespace cd
