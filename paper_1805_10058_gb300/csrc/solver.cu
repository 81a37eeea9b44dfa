// Solver handle, Krylov orchestration (FP64 PCG, FP32-inner / FP64 iterative refinement),
// preconditioners and the C-ABI entry points of include/curldiv.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <memory>
#include <mutex>
#include <tuple>

#include "krylov.h"
#include "mg.h"

namespace cd {
uint64_t launches();
int launch_symbol_eigs(int d, int p, double alpha, double beta, const double* nu, int mg,
                       double* lam, double* lap, cudaStream_t s);
void lanczos_run(long long N, int B, int steps, const double* v0, double* v, double* w,
                 double* vprev, double* la, double* lb, double* coef, double* inv, int* live,
                 int* used, double* part, void (*apply)(void*, const double*, double*), void* ctx,
                 cudaStream_t s);
void tridiag_extremes(const double* a, const double* b, int k, double* lmin, double* lmax);

// ------------------------------------------------------------------ device buffers
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t b) {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = b;
    return b ? cudaMalloc(&p, b) : cudaSuccess;
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

template <typename T>
static cudaError_t upload(DevBuf& d, const std::vector<T>& h) {
  cudaError_t e = d.alloc(h.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}
template <typename T>
static std::vector<T> cast_vec(const std::vector<double>& v) {
  std::vector<T> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (T)v[i];
  return o;
}

struct Workspace {  // one precision's Krylov vectors
  DevBuf x, r, z, p, q, zold, fa, fb, mg;
  DevBuf apply_scratch;
};

}  // namespace cd

using namespace cd;

struct cd_solver_s {
  int d = 0, p = 0, n = 0, m = 0, P = 0;
  // anisotropic mesh (Section 5): ma[l] unknowns per component along x_l; bands of direction l
  // at aoff[l] in bands64 / bands32 ([3][ma[l]][2P+1] row-major); FD-D eigenbases per direction
  bool aniso = false;
  int ma[3] = {0, 0, 0};
  size_t aoff[3] = {0, 0, 0};
  DevBuf aU64, aUt64, alam64, aU32, aUt32, alam32;  // per direction, concatenated
  size_t aUoff[3] = {0, 0, 0}, alamoff[3] = {0, 0, 0};
  double alpha0 = 1, beta0 = 1;
  cd_options opt{};
  cudaStream_t s = nullptr;
  long long N = 0;  // DoF per RHS
  int Bcap = 0;
  std::vector<Band> hM, hA, hS;  // per level
  std::vector<int> ml;           // per-level m
  DevBuf bands64, bands32;       // all levels concatenated: level l at offset boff[l]
  std::vector<size_t> boff;
  // FD eigenbases (finest level)
  std::vector<double> UD, lamD, UT, lamT;
  DevBuf UD64, UDt64, lamD64, UT64, UTt64, lamT64, UD32, UDt32, lamD32, UT32, UTt32, lamT32;
  bool have_fd = false;
  // banded Cholesky factor of T_m (off-diagonal taps, inverse diagonal), built on first need
  DevBuf TB64, TBd64, TB32, TBd32;
  bool have_tband = false;
  // per-solve coefficients and state
  DevBuf alpha, beta;
  DevBuf sd[6];  // rz rr rr0 alpha beta rzold
  DevBuf si[3];  // active iters status
  DevBuf sd2[6], si2[3];  // a second PCG state: the FP64 inner group of a serving session
  // serving session (iteration-level continuous batching): per-slot phase (0 free, 1 pending
  // admission, 2 outer step due, 3 FP32 inner solve, 4 FP64 inner solve, 5 finished), right-hand
  // sides and solutions [B][N], device masks, parameters
  std::vector<int> sp;
  std::vector<double> s_alpha, s_beta;
  std::vector<std::chrono::steady_clock::time_point> s_t0;
  DevBuf s_b, s_x, s_mask;  // s_mask: 4 int arrays [B]
  std::vector<int> h_mask;
  DevBuf part[4];
  DevBuf ir_rnorm, ir_bnorm2, ir_relres, ir_active, ir_status, ir_outer, ir_inner_total, cnt;
  DevBuf ir_rrprev, ir_grp, ir_tol2, ir_m0, ir_m1, ir_m2;
  DevBuf b64, x64, r64;
  DevBuf xlo64, ext_scratch;  // low parts of the double-FP64 solution; residual intermediates
  DevBuf lz_a, lz_b;          // Lanczos tridiagonal coefficients (cd_lanczos)
  int ext_chunk = 0;          // solves per launch of the extended residual
  Workspace w64, w32;
  int* h_cnt = nullptr;  // pinned
  MgData mg;
  std::vector<double> mg_alpha, mg_beta;  // parameters the multigrid data was prepared for
  MgData mgD;                               // hierarchy of the block diagonal D (P_WL)
  bool have_mgD = false;
  std::vector<double> mgD_alpha, mgD_beta;
  std::vector<double> dev_alpha, dev_beta;  // host mirror of the per-solve alpha, beta on the device
  // CUDA graphs of a chunk of PCG iterations, keyed by (f32, B, pc, flexible, arithmetic
  // flags, maxit, PCG state)
  std::map<std::tuple<int, int, int, int, int, int, int>, std::pair<cudaGraphExec_t, uint64_t>> graphs;
  std::mutex mu;
  ~cd_solver_s() {
    for (size_t l = 0; l < boff.size(); ++l) {
      if (bands64.p) unregister_level(bands64.as<double>() + boff[l]);
      if (bands32.p) unregister_level(bands32.as<float>() + boff[l]);
    }
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.first);
    if (h_cnt) cudaFreeHost(h_cnt);
  }
};

namespace cd {

// PCG state 0 (every solve of a batched call; the FP32 group of a session) or 1 (the FP64 group
// of a session, which runs interleaved with the FP32 one)
static PcgState state_of(cd_solver h, int which = 0) {
  DevBuf* sd = which ? h->sd2 : h->sd;
  DevBuf* si = which ? h->si2 : h->si;
  PcgState st;
  st.rz = sd[0].as<double>();
  st.rr = sd[1].as<double>();
  st.rr0 = sd[2].as<double>();
  st.alpha = sd[3].as<double>();
  st.beta = sd[4].as<double>();
  st.rzold = sd[5].as<double>();
  st.active = si[0].as<int>();
  st.iters = si[1].as<int>();
  st.status = si[2].as<int>();
  return st;
}

template <typename T>
static const T* bands_of(cd_solver h, int level) {
  if (sizeof(T) == 8) return reinterpret_cast<const T*>(h->bands64.as<double>() + h->boff[level]);
  return reinterpret_cast<const T*>(h->bands32.as<float>() + h->boff[level]);
}
template <typename T>
static Workspace& ws_of(cd_solver h) {
  return sizeof(T) == 8 ? h->w64 : h->w32;
}

static Coef coef_of(cd_solver h) { return Coef{h->alpha.as<double>(), h->beta.as<double>()}; }

template <typename T>
static int apply_level(cd_solver h, int level, const T* w, T* y, const T* rhs, int mode, int B,
                       double* dotp, int* nblk, const int* active) {
  if (h->aniso) {
    const T* base = sizeof(T) == 8 ? (const T*)h->bands64.p : (const T*)h->bands32.p;
    const T* band[3] = {base + h->aoff[0], base + h->aoff[1], base + h->aoff[2]};
    return launch_apply_aniso<T>(h->d, h->ma, h->P, band, w, y, rhs, mode, B, coef_of(h), dotp,
                                 nblk, active, ws_of<T>(h).apply_scratch.template as<T>(), h->s);
  }
  return launch_apply<T>(h->d, h->ml[level], h->P, bands_of<T>(h, level), w, y, rhs, mode, B,
                         coef_of(h), dotp, nblk, active,
                         ws_of<T>(h).apply_scratch.template as<T>(), h->s);
}

// One FD pass: FP32 on tcgen05 when enabled (all solves of the batch), else SIMT.
template <typename T>
static void fd_pass(cd_solver h, int axis, int B, const T* G, const T* in, T* out, FdScale<T> sc,
                    const int* active) {
  if (sizeof(T) == 4 && h->opt.fd_tensor_cores &&
      launch_fd_axis_tc(h->d, h->m, axis, B, (const float*)G, (const float*)in, (float*)out,
                        *reinterpret_cast<FdScale<float>*>(&sc), h->s))
    return;
  launch_fd_axis<T>(h->d, h->m, axis, B, G, in, out, sc, active, h->s);
}

// The inner FP64 solves of a mixed-precision solve apply a fast-diagonalisation preconditioner
// in FP32 (tensor-core transforms): a preconditioner needs no FP64 accuracy, and the FP64 FD
// passes run on GB300's narrow FP64 pipe.  Set by the refinement loop for its FP64 group.
static thread_local int g_lowp_prec = 0;

template <typename T>
static void apply_prec(cd_solver h, int pc, int B, const T* r, T* z, const int* active);

// z = B^{-1} r for an FD preconditioner of an FP64 solve, computed in FP32
static void apply_fd_lowp(cd_solver h, int pc, int B, const double* r, double* z, const int* active) {
  Workspace& w = ws_of<float>(h);
  to_f32(h->N, B, r, w.r.as<float>(), active, h->s);
  apply_prec<float>(h, pc, B, w.r.as<float>(), w.z.as<float>(), active);
  to_f64(h->N, B, w.z.as<float>(), z, active, h->s);
}

// z = B^{-1} r for the preconditioner kind pc.
template <typename T>
static void apply_prec(cd_solver h, int pc, int B, const T* r, T* z, const int* active) {
  Workspace& w = ws_of<T>(h);
  if constexpr (sizeof(T) == 8) {
    if (g_lowp_prec && (pc == CD_PC_FD_D || pc == CD_PC_FD_T)) {
      apply_fd_lowp(h, pc, B, r, z, active);
      return;
    }
  }
  if (pc == CD_PC_NONE) {
    vcopy<T>(h->N, B, r, z, active, h->s);
    return;
  }
  if (h->aniso) {  // FD-D with the eigenbases of each direction (the only other kind offered)
    const bool f64 = sizeof(T) == 8;
    const T* U = (const T*)(f64 ? h->aU64.p : h->aU32.p);
    const T* Ut = (const T*)(f64 ? h->aUt64.p : h->aUt32.p);
    const T* L = (const T*)(f64 ? h->alam64.p : h->alam32.p);
    const T* lam[3] = {L + h->alamoff[0], L + h->alamoff[1], L + h->alamoff[2]};
    T* bufs[2] = {w.fa.as<T>(), w.fb.as<T>()};
    const T* src = r;
    int pass = 0;
    for (int a = h->d - 1; a >= 0; --a, ++pass) {  // U_l^T along every direction
      launch_fd_axis_aniso<T>(h->d, h->ma, a, B, U + h->aUoff[a], src, bufs[pass & 1], active, h->s);
      src = bufs[pass & 1];
    }
    launch_fd_scale_aniso<T>(h->d, h->ma, lam, B, h->alpha.as<double>(), h->beta.as<double>(),
                             bufs[(pass - 1) & 1], active, h->s);
    for (int a = h->d - 1; a >= 0; --a, ++pass) {  // U_l along every direction
      T* dst = a == 0 ? z : bufs[pass & 1];
      launch_fd_axis_aniso<T>(h->d, h->ma, a, B, Ut + h->aUoff[a], src, dst, active, h->s);
      src = dst;
    }
    return;
  }
  if (pc == CD_PC_MG) {
    mg_vcycle<T>(h->mg, h->d, h->P, B, r, z, coef_of(h), active, h->s, w.apply_scratch.as<T>());
    return;
  }
  if (pc == CD_PC_MIM) {  // P_MIM: two V-cycles, PGMRES-T post-smoothing on the finest level
    mg_vcycle<T>(h->mg, h->d, h->P, B, r, z, coef_of(h), active, h->s, w.apply_scratch.as<T>(),
                 kPostPgmres, 2);
    return;
  }
  if (pc == CD_PC_WL) {  // P_WL: one V-cycle on D, PCG-T post-smoothing on the finest level
    mg_vcycle<T>(h->mgD, h->d, h->P, B, r, z, coef_of(h), active, h->s, w.apply_scratch.as<T>(),
                 kPostPcg, 1);
    return;
  }
  if (pc == CD_PC_T_BAND) {
    const T* Lb = (const T*)(sizeof(T) == 8 ? h->TB64.p : h->TB32.p);
    const T* dinv = (const T*)(sizeof(T) == 8 ? h->TBd64.p : h->TBd32.p);
    launch_tband<T>(h->d, h->m, h->p - 1, B, Lb, dinv, r, z, active, h->s);
    return;
  }
  const bool isD = pc == CD_PC_FD_D;
  const T *U, *Ut, *lam;
  if (sizeof(T) == 8) {
    U = (const T*)(isD ? h->UD64.p : h->UT64.p);
    Ut = (const T*)(isD ? h->UDt64.p : h->UTt64.p);
    lam = (const T*)(isD ? h->lamD64.p : h->lamT64.p);
  } else {
    U = (const T*)(isD ? h->UD32.p : h->UT32.p);
    Ut = (const T*)(isD ? h->UDt32.p : h->UTt32.p);
    lam = (const T*)(isD ? h->lamD32.p : h->lamT32.p);
  }
  const int d = h->d, m = h->m;
  T* bufs[2] = {w.fa.as<T>(), w.fb.as<T>()};
  const T* src = r;
  int pass = 0;
  for (int a = d - 1; a >= 0; --a) {  // forward: U^T along every axis, then scale
    T* dst = bufs[pass & 1];
    FdScale<T> sc{};
    if (a == 0) {
      sc.mode = isD ? 1 : 2;
      sc.d = d;
      sc.m = m;
      sc.per = h->N / d;
      sc.lam = lam;
      sc.alpha = h->alpha.as<double>();
      sc.beta = h->beta.as<double>();
      sc.base = dst;
    }
    fd_pass<T>(h, a, B, U, src, dst, sc, active);
    src = dst;
    ++pass;
  }
  for (int a = d - 1; a >= 0; --a) {  // backward: U along every axis
    T* dst = (a == 0) ? z : bufs[pass & 1];
    fd_pass<T>(h, a, B, Ut, src, dst, FdScale<T>{}, active);
    src = dst;
    ++pass;
  }
}

// One PCG iteration (all kernels masked by the per-solve active flags).
template <typename T>
static void pcg_iteration(cd_solver h, int B, int pc, int flexible, const double* tol2v, int maxit,
                          int which = 0) {
  Workspace& w = ws_of<T>(h);
  PcgState st = state_of(h, which);
  const long long N = h->N;
  const int nb = partial_blocks(N);
  int npq = 0;
  apply_level<T>(h, 0, w.p.as<T>(), w.q.as<T>(), nullptr, 0, B, h->part[0].as<double>(), &npq,
                 st.active);
  cg_alpha(B, st, h->part[0].as<double>(), npq, h->s);
  cg_update<T>(N, B, nb, w.x.as<T>(), w.r.as<T>(), w.p.as<T>(), w.q.as<T>(),
               flexible ? w.z.as<T>() : nullptr, st.alpha, st.active, h->part[1].as<double>(),
               h->part[2].as<double>(), h->s);
  cg_check(B, st, h->part[1].as<double>(), nb, flexible ? h->part[2].as<double>() : nullptr, nb,
           tol2v, maxit, h->s);
  apply_prec<T>(h, pc, B, w.r.as<T>(), w.z.as<T>(), st.active);
  launch_dot<T>(w.r.as<T>(), w.z.as<T>(), N, B, h->part[3].as<double>(), nb, st.active, h->s);
  cg_beta(B, st, h->part[3].as<double>(), nb, flexible, h->s);
  xpay<T>(N, B, w.z.as<T>(), w.p.as<T>(), st.beta, st.active, h->s);
}

// Starts PCG on the workspace of precision T for the solves in `outer_active`: r holds the
// right-hand side, x = 0, z = M r, p = z and the per-solve scalars of PCG state `which`; with
// keep_others the other solves' state is left untouched (a session's solves mid-way through
// their own PCG), else they are stopped.  Returns whether the method is flexible.
template <typename T>
static int pcg_begin(cd_solver h, int B, int pc, const int* outer_active, int which,
                     int keep_others = 0) {
  Workspace& w = ws_of<T>(h);
  PcgState st = state_of(h, which);
  const long long N = h->N;
  const int nb = partial_blocks(N);
  // a Krylov-smoothed / multigrid or tensor-core (TF32) preconditioner is not an exactly
  // fixed symmetric operator: use the flexible update there
  const bool fd = pc == CD_PC_FD_D || pc == CD_PC_FD_T;
  const int flexible = (pc == CD_PC_MG || pc == CD_PC_MIM || pc == CD_PC_WL ||
                        (sizeof(T) == 4 && h->opt.fd_tensor_cores && fd) ||
                        (sizeof(T) == 8 && g_lowp_prec && fd))
                           ? 1
                           : 0;
  vzero<T>(N, B, w.x.as<T>(), outer_active, h->s);
  apply_prec<T>(h, pc, B, w.r.as<T>(), w.z.as<T>(), outer_active);
  launch_dot<T>(w.r.as<T>(), w.r.as<T>(), N, B, h->part[1].as<double>(), nb, outer_active, h->s);
  launch_dot<T>(w.r.as<T>(), w.z.as<T>(), N, B, h->part[3].as<double>(), nb, outer_active, h->s);
  cg_init(B, st, h->part[1].as<double>(), nb, h->part[3].as<double>(), nb, outer_active, h->s,
          keep_others);
  vcopy<T>(N, B, w.z.as<T>(), w.p.as<T>(), outer_active, h->s);
  return flexible;
}

// Enqueues one chunk of opt.chunk PCG iterations of state `which` (a CUDA graph when enabled)
// followed by the count of its still-active solves into cnt[0].
template <typename T>
static cd_status pcg_chunk(cd_solver h, int B, int pc, int flexible, const double* tol2v, int maxit,
                           int which) {
  PcgState st = state_of(h, which);
  const int chunk = std::max(1, h->opt.chunk);
  cudaGraphExec_t exec = nullptr;
  uint64_t nodes = 0;
  if (h->opt.use_graphs) {
    auto key = std::make_tuple((int)(sizeof(T) == 4), B, pc, flexible,
                               fp64_emulated() + 2 * g_lowp_prec, maxit, which);
    auto it = h->graphs.find(key);
    if (it != h->graphs.end()) {
      exec = it->second.first;
      nodes = it->second.second;
    } else {
      cudaGraph_t g = nullptr;
      const uint64_t c0 = launches();
      if (cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        for (int k = 0; k < chunk; ++k) pcg_iteration<T>(h, B, pc, flexible, tol2v, maxit, which);
        count_active(B, st.active, h->cnt.as<int>(), h->s);
        if (cudaStreamEndCapture(h->s, &g) == cudaSuccess && g) {
          if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
          cudaGraphDestroy(g);
        }
      }
      nodes = launches() - c0;
      count_launch(-(int)nodes);  // captured, not launched
      cudaGetLastError();
      if (exec) h->graphs[key] = std::make_pair(exec, nodes);
    }
  }
  if (exec) {
    CD_CUDA_OK(cudaGraphLaunch(exec, h->s));
    count_launch((int)nodes);
  } else {
    for (int k = 0; k < chunk; ++k) pcg_iteration<T>(h, B, pc, flexible, tol2v, maxit, which);
    count_active(B, st.active, h->cnt.as<int>(), h->s);
  }
  return CD_OK;
}

// Runs PCG on the workspace of precision T: r holds the right-hand side on entry, x the
// solution on exit (x_0 = 0).  outer_active masks the solves that take part.
template <typename T>
static cd_status run_pcg(cd_solver h, int B, int pc, const double* tol2v, int maxit,
                         const int* outer_active) {
  const int flexible = pcg_begin<T>(h, B, pc, outer_active, 0);
  const int chunk = std::max(1, h->opt.chunk);
  for (int done = 0; done < maxit + chunk; done += chunk) {
    cd_status st = pcg_chunk<T>(h, B, pc, flexible, tol2v, maxit, 0);
    if (st != CD_OK) return st;
    CD_CUDA_OK(cudaMemcpyAsync(h->h_cnt, h->cnt.p, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CD_CUDA_OK(cudaStreamSynchronize(h->s));
    if (*h->h_cnt == 0) break;
  }
  CD_CUDA_OK(cudaGetLastError());
  return CD_OK;
}

__global__ void add_iters_kernel(int B, const int* iters, const int* active, int* total) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B && active[b]) total[b] += iters[b];
}
__global__ void set_int_kernel(int B, int* a, int v) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) a[b] = v;
}
__global__ void d2f_kernel(long long n, const double* a, float* b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void f2d_kernel(long long n, const float* a, double* b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// Outer residual r64 = b - A (x + xlo) with per-solve partial sums of r^T r in part[0]
// (*npart partials per solve): double-FP64 when the handle keeps an extended solution (xlo
// may then be NULL for the FP64 x alone), else the FP64 apply in residual mode.
static cd_status outer_residual(cd_solver h, int B, const double* b, const double* x,
                                const double* xlo, const int* active, int* npart) {
  if (h->opt.ext_residual) {
    if (launch_ext_residual(h->d, h->m, h->P, bands_of<double>(h, 0), b, x, xlo,
                            h->r64.as<double>(), B, coef_of(h), active,
                            h->ext_scratch.as<double>(), h->ext_chunk, h->s) != 0) {
      set_error("extended residual: unsupported shape");
      return CD_EINVAL;
    }
    *npart = partial_blocks(h->N);
    launch_dot<double>(h->r64.as<double>(), h->r64.as<double>(), h->N, B, h->part[0].as<double>(),
                       *npart, active, h->s);
    return CD_OK;
  }
  apply_level<double>(h, 0, x, h->r64.as<double>(), b, 1, B, h->part[0].as<double>(), npart,
                      active);
  return CD_OK;
}

// Final ||b - A x|| / ||b|| per solve for reporting (same evaluation as the outer loop).
static cd_status final_residual(cd_solver h, int B, const double* b, const double* x,
                                const double* xlo, std::vector<double>& relres) {
  const int nb = partial_blocks(h->N);
  int npart = 0;
  cd_status st = outer_residual(h, B, b, x, xlo, nullptr, &npart);
  if (st != CD_OK) return st;
  launch_dot<double>(b, b, h->N, B, h->part[1].as<double>(), nb, nullptr, h->s);
  std::vector<double> prr((size_t)B * npart), pbb((size_t)B * nb);
  CD_CUDA_OK(cudaMemcpyAsync(prr.data(), h->part[0].p, prr.size() * 8, cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaMemcpyAsync(pbb.data(), h->part[1].p, pbb.size() * 8, cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaStreamSynchronize(h->s));
  relres.assign(B, 0.0);
  for (int i = 0; i < B; ++i) {
    double rr = 0, bb = 0;
    for (int k = 0; k < npart; ++k) rr += prr[(size_t)i * npart + k];
    for (int k = 0; k < nb; ++k) bb += pbb[(size_t)i * nb + k];
    relres[i] = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  }
  return CD_OK;
}

static cd_status set_params(cd_solver h, int nrhs, const double* alphas, const double* betas,
                            std::vector<double>* pa = nullptr, std::vector<double>* pb = nullptr,
                            int pc_kind = -1) {
  std::vector<double> a(nrhs), b(nrhs);
  for (int i = 0; i < nrhs; ++i) {
    a[i] = alphas ? alphas[i] : h->alpha0;
    b[i] = betas ? betas[i] : h->beta0;
    if (!(a[i] > 0) || !(b[i] > 0) || !std::isfinite(a[i]) || !std::isfinite(b[i])) {
      set_error("alpha and beta must be finite and > 0");
      return CD_EINVAL;
    }
  }
  // upload only what changed since the last call (a repeated apply or solve with the same
  // parameters then launches its kernels without a copy or a host synchronisation)
  const bool same = (int)h->dev_alpha.size() >= nrhs &&
                    std::equal(a.begin(), a.end(), h->dev_alpha.begin()) &&
                    std::equal(b.begin(), b.end(), h->dev_beta.begin());
  if (!same) {
    CD_CUDA_OK(cudaMemcpyAsync(h->alpha.p, a.data(), nrhs * 8, cudaMemcpyHostToDevice, h->s));
    CD_CUDA_OK(cudaMemcpyAsync(h->beta.p, b.data(), nrhs * 8, cudaMemcpyHostToDevice, h->s));
    CD_CUDA_OK(cudaStreamSynchronize(h->s));  // a, b are stack vectors
    if ((int)h->dev_alpha.size() < nrhs) {
      h->dev_alpha.resize(nrhs);
      h->dev_beta.resize(nrhs);
    }
    std::copy(a.begin(), a.end(), h->dev_alpha.begin());
    std::copy(b.begin(), b.end(), h->dev_beta.begin());
  }
  if (pa) *pa = a;
  if (pb) *pb = b;
  if (pc_kind == CD_PC_WL && (a != h->mgD_alpha || b != h->mgD_beta)) {
    cd_status st = mg_set_params(h->mgD, h->d, h->P, nrhs, a, b, h->s);
    if (st != CD_OK) return st;
    st = mg_prepare(h->mgD, nrhs, coef_of(h), h->w64.apply_scratch.as<double>(), h->s);
    if (st != CD_OK) return st;
    h->mgD_alpha = a;
    h->mgD_beta = b;
  }
  const bool need_mg = pc_kind == CD_PC_MG || pc_kind == CD_PC_MIM;
  if (need_mg && (a != h->mg_alpha || b != h->mg_beta)) {
    cd_status st = mg_set_params(h->mg, h->d, h->P, nrhs, a, b, h->s);
    if (st != CD_OK) return st;
    st = mg_prepare(h->mg, nrhs, coef_of(h), h->w64.apply_scratch.as<double>(), h->s);
    if (st != CD_OK) return st;
    h->mg_alpha = a;  // Chebyshev bounds and coarse inverses now match these parameters
    h->mg_beta = b;
  }
  return CD_OK;
}

// Solves A x = b for B right-hand sides.  With ext_residual the solution is carried as
// x + xlo (double-FP64); `xlo_out` (may be NULL) receives the low part and decides which
// solution the status and relres describe: x + xlo when given, x alone otherwise.
static cd_status solve_device(cd_solver h, const double* b, double* x, double* xlo_out, int B,
                              cd_result* res, const std::vector<double>& alphas,
                              const std::vector<double>& betas) {
  auto t0 = std::chrono::steady_clock::now();
  const long long N = h->N;
  const int pc = h->opt.precond;
  std::vector<int> status(B, CD_OK), inner(B, 0), outer(B, 1);
  // inner precision group per solve: 0 = FP32 Krylov + FP32 preconditioner, 2 = all FP64
  // (group 1 is unused: an FP32 preconditioner inside FP64 Krylov was measured to need
  // several times more iterations than FP64 throughout at parameter ratios of 1e6)
  std::vector<int> grp(B, 2);
  if (h->opt.precision == CD_PREC_FP32_IR)
    for (int i = 0; i < B; ++i) {
      const double ratio = std::max(alphas[i], betas[i]) / std::min(alphas[i], betas[i]);
      grp[i] = ratio >= h->opt.mixed_switch_ratio ? 2 : 0;
    }
  const int nb = partial_blocks(N);
  int* act = h->ir_active.as<int>();
  int* m[3] = {h->ir_m0.as<int>(), h->ir_m1.as<int>(), h->ir_m2.as<int>()};
  CD_CUDA_OK(cudaMemcpyAsync(h->ir_grp.p, grp.data(), B * 4, cudaMemcpyHostToDevice, h->s));
  set_int_kernel<<<(B + 127) / 128, 128, 0, h->s>>>(B, act, 1);
  set_int_kernel<<<(B + 127) / 128, 128, 0, h->s>>>(B, h->ir_status.as<int>(), CD_NOT_CONVERGED);
  set_int_kernel<<<(B + 127) / 128, 128, 0, h->s>>>(B, h->ir_outer.as<int>(), 0);
  set_int_kernel<<<(B + 127) / 128, 128, 0, h->s>>>(B, h->ir_inner_total.as<int>(), 0);
  count_launch(4);
  vzero<double>(N, B, x, nullptr, h->s);
  const bool ext = h->opt.ext_residual != 0;
  // Mixed precision: the FP64 inner solves apply the operator in double-FP32 on the FP32 pipe
  // (2D: the packed folded kernel; 3D: the tuned passes with (hi, lo) intermediates), and the
  // double-FP64 outer residual corrects its coarser rounding.  CD_PREC_FP64 keeps FP64
  // arithmetic throughout.
  const bool emu_inner = ext && h->opt.emulated_fp64 && h->opt.precision != CD_PREC_FP64;
  double* xlo = ext ? h->xlo64.as<double>() : nullptr;
  if (ext) vzero<double>(N, B, xlo, nullptr, h->s);
  launch_dot<double>(b, b, N, B, h->part[1].as<double>(), nb, nullptr, h->s);
  launch_sum_partials(h->part[1].as<double>(), nb, B, h->ir_bnorm2.as<double>(), h->s);
  const double inner2 = h->opt.inner_rtol * h->opt.inner_rtol;
  const double* tol2v = h->ir_tol2.as<double>();
  for (int step = 0; step <= h->opt.max_outer + 1; ++step) {
    int npart = 0;
    cd_status rst = outer_residual(h, B, b, x, xlo, act, &npart);
    if (rst != CD_OK) return rst;
    ir_check(B, h->part[0].as<double>(), npart, h->ir_bnorm2.as<double>(), h->ir_rnorm.as<double>(),
             h->ir_rrprev.as<double>(), act, h->ir_status.as<int>(), h->ir_relres.as<double>(),
             h->ir_outer.as<int>(), h->ir_grp.as<int>(), h->ir_tol2.as<double>(),
             h->opt.rtol * h->opt.rtol, inner2, h->opt.max_outer, h->ir_inner_total.as<int>(),
             h->opt.maxit, emu_inner ? 1e-12 : 1e-30, h->s);
    group_masks(B, act, h->ir_grp.as<int>(), m[0], m[1], m[2], h->cnt.as<int>(), h->s);
    CD_CUDA_OK(cudaMemcpyAsync(h->h_cnt, h->cnt.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CD_CUDA_OK(cudaStreamSynchronize(h->s));
    int cnt[4] = {h->h_cnt[0], h->h_cnt[1], h->h_cnt[2], h->h_cnt[3]};
    if (cnt[3] == 0) break;
    if (cnt[0] > 0) {
      ir_cast(N, B, h->r64.as<double>(), h->w32.r.as<float>(), h->ir_rnorm.as<double>(), m[0], h->s);
      cd_status st = run_pcg<float>(h, B, pc, tol2v, h->opt.inner_maxit, m[0]);
      if (st != CD_OK) return st;
      add_iters_kernel<<<(B + 127) / 128, 128, 0, h->s>>>(B, h->si[1].as<int>(), m[0],
                                                          h->ir_inner_total.as<int>());
      count_launch();
      if (ext)
        launch_ext_update<float>(N, B, x, xlo, h->w32.x.as<float>(), h->ir_rnorm.as<double>(), m[0],
                                 h->s);
      else
        ir_update(N, B, x, h->w32.x.as<float>(), h->ir_rnorm.as<double>(), m[0], h->s);
    }
    for (int g = 1; g <= 2; ++g) {
      if (cnt[g] == 0) continue;
      scale_div(N, B, h->r64.as<double>(), h->w64.r.as<double>(), h->ir_rnorm.as<double>(), m[g], h->s);
      // the first FP64 inner solve may use the whole budget.  With an FP64 outer residual a
      // restart only has to correct the drift of the recursive residual (or show that the FP64
      // floor is reached); with the double-FP64 residual it continues below that floor and
      // keeps the whole budget (the outer check stops a solve at maxit iterations in total).
      const int cap = (step == 0 || ext) ? h->opt.maxit
                                         : std::min({h->opt.maxit, h->opt.inner_maxit, 500});
      set_fp64_emulated(emu_inner ? 1 : 0);
      g_lowp_prec = h->opt.precision == CD_PREC_FP32_IR ? 1 : 0;
      cd_status st = run_pcg<double>(h, B, pc, tol2v, cap, m[g]);
      set_fp64_emulated(0);
      g_lowp_prec = 0;
      if (st != CD_OK) return st;
      add_iters_kernel<<<(B + 127) / 128, 128, 0, h->s>>>(B, h->si[1].as<int>(), m[g],
                                                          h->ir_inner_total.as<int>());
      count_launch();
      if (ext)
        launch_ext_update<double>(N, B, x, xlo, h->w64.x.as<double>(), h->ir_rnorm.as<double>(),
                                  m[g], h->s);
      else
        ir_update64(N, B, x, h->w64.x.as<double>(), h->ir_rnorm.as<double>(), m[g], h->s);
    }
  }
  CD_CUDA_OK(cudaMemcpyAsync(status.data(), h->ir_status.p, B * 4, cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaMemcpyAsync(inner.data(), h->ir_inner_total.p, B * 4, cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaMemcpyAsync(outer.data(), h->ir_outer.p, B * 4, cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaStreamSynchronize(h->s));
  if (fd_tc_error()) {
    set_error("a tensor-core FD kernel gave up waiting for its MMAs");
    return CD_ECUDA;
  }
  // x = the FP64 rounding of x + xlo already (the update renormalises the pair)
  std::vector<double> rel_hi, rel_ext;
  cd_status st = final_residual(h, B, b, x, nullptr, rel_hi);
  if (st != CD_OK) return st;
  if (ext && xlo_out) {
    st = final_residual(h, B, b, x, xlo, rel_ext);
    if (st != CD_OK) return st;
  } else {
    rel_ext = rel_hi;
  }
  if (xlo_out) {
    if (ext)
      CD_CUDA_OK(cudaMemcpyAsync(xlo_out, xlo, 8 * (size_t)B * N, cudaMemcpyDeviceToDevice, h->s));
    else
      vzero<double>(N, B, xlo_out, nullptr, h->s);
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  cd_status worst = CD_OK;
  for (int i = 0; i < B; ++i) {
    int s_i = status[i];
    // the status describes the solution returned: x + xlo when the caller takes xlo
    const double rel = xlo_out ? rel_ext[i] : rel_hi[i];
    if (s_i == CD_OK && !(rel <= h->opt.rtol)) s_i = CD_NOT_CONVERGED;
    if (s_i != CD_OK && worst == CD_OK) worst = (cd_status)s_i;
    if (res) {
      res[i].iters_outer = outer[i];
      res[i].iters_inner = inner[i];
      res[i].relres = rel;
      res[i].relres_hi = rel_hi[i];
      res[i].seconds = secs;
      res[i].status = s_i;
    }
  }
  if (xlo_out) CD_CUDA_OK(cudaStreamSynchronize(h->s));
  return worst;
}

}  // namespace cd

namespace cd {
// FD eigenbases of the finest level (generalized for D, symmetric for T); built on first need.
static cd_status ensure_fd(cd_solver h) {
  if (h->have_fd) return CD_OK;
  const int m = h->m, p = h->p, P = h->P;
    std::vector<double> Md = band_to_dense(h->hM[0]), Sd = band_to_dense(h->hS[0]);
    if (!gen_eig(m, Md, Sd, h->UD, h->lamD)) {
      set_error("generalized eigen-decomposition failed");
      return CD_EINVAL;
    }
    Band T;
    toeplitz_T_band(p, m, P, T);
    std::vector<double> Td = band_to_dense(T);
    sym_eig(m, Td, h->UT, h->lamT);
    auto transpose = [m](const std::vector<double>& U) {
      std::vector<double> t((size_t)m * m);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) t[(size_t)j * m + i] = U[(size_t)i * m + j];
      return t;
    };
    std::vector<double> UDt = transpose(h->UD), UTt = transpose(h->UT);
    bool ok = upload(h->UD64, h->UD) == cudaSuccess && upload(h->UDt64, UDt) == cudaSuccess &&
              upload(h->lamD64, h->lamD) == cudaSuccess && upload(h->UT64, h->UT) == cudaSuccess &&
              upload(h->UTt64, UTt) == cudaSuccess && upload(h->lamT64, h->lamT) == cudaSuccess &&
              upload(h->UD32, cast_vec<float>(h->UD)) == cudaSuccess &&
              upload(h->UDt32, cast_vec<float>(UDt)) == cudaSuccess &&
              upload(h->lamD32, cast_vec<float>(h->lamD)) == cudaSuccess &&
              upload(h->UT32, cast_vec<float>(h->UT)) == cudaSuccess &&
              upload(h->UTt32, cast_vec<float>(UTt)) == cudaSuccess &&
              upload(h->lamT32, cast_vec<float>(h->lamT)) == cudaSuccess;
    if (!ok) {
      set_error("eigenbasis upload failed");
      return CD_ECUDA;
    }
    h->have_fd = true;
  return CD_OK;
}
}  // namespace cd

namespace cd {
// Device bytes a handle for (d, p, n) allocates with these options (the estimate the serving
// runtime admits against; it mirrors the allocations of cd_create and mg_build).
// Coarsest multigrid size: the option, or (0) 16 for the Chebyshev multigrid in 2D (a dense
// coarse solve of at most 2 * 16^2 unknowns replaces three launch-bound levels) and 3 otherwise
// (the paper's strategies P_MIM / P_WL keep its hierarchy, Section 6.1, down to m <= 3).
static int mg_coarsest(int d, int opt_m_min, int precond) {
  if (opt_m_min <= 0) return d == 2 && precond == CD_PC_MG ? 16 : 3;
  return opt_m_min;
}

size_t solver_bytes(int d, int p, int n, const cd_options& opt) {
  const size_t B = (size_t)std::max(1, opt.max_batch);
  const size_t N = cd_dofs(d, p, n);
  const int m = n + p - 2, W = 2 * p + 1;
  size_t bytes = 0;
  size_t nl = 0, n3 = 0, n3_1 = 0, nc = 0;
  for (int ml = m, l = 0;; ++l) {
    nl += 2 * (size_t)3 * ml * W + 8;  // bands of the level
    if (l == 0) n3 = (size_t)ml * ml * ml;
    if (l == 1) n3_1 = (size_t)ml * ml * ml;
    nc = d == 2 ? (size_t)2 * ml * ml : (size_t)3 * ml * ml * ml;
    if (ml <= mg_coarsest(d, opt.mg_m_min, opt.precond) || ml / 2 < 1) break;
    ml /= 2;
  }
  bytes += nl * 12;
  bytes += B * nc * nc * 12;  // dense coarsest inverses (FP64 and FP32) per solve
  bytes += B * N * (7 * 8 + 7 * 4 + 8 + 16);  // Krylov workspaces, r64, b64/x64
  if (d == 3) bytes += 21 * n3 * B * 12;
  bytes += 4 * 8 * B * kMaxPartials + 64 * B;
  // multigrid levels: five vectors per level and precision (level sizes shrink by 2^d)
  bytes += (size_t)(5 * 12 * (double)B * N * (d == 2 ? 4.0 / 3.0 : 8.0 / 7.0));
  if (d == 3) bytes += 21 * n3_1 * B * 12;
  if (opt.precond == CD_PC_FD_D || opt.precond == CD_PC_FD_T)
    bytes += (size_t)m * m * 12 * 4;
  if (opt.precond == CD_PC_MIM || opt.precond == CD_PC_WL) {
    bytes += B * N * (2 * (size_t)p + 4) * 12;  // Krylov smoother and cycle vectors
    if (opt.precond == CD_PC_WL)                 // the second (block-diagonal) hierarchy
      bytes += (size_t)(6 * 12 * (double)B * N * (d == 2 ? 4.0 / 3.0 : 8.0 / 7.0));
  }
  if (opt.ext_residual) {
    const size_t per = (size_t)6 * N;  // residual intermediates (hi, lo) per solve, doubles
    bytes += 8 * B * N + 8 * std::min(B * per, std::max(per, (size_t)(256u << 20) / 8));
  }
  return (size_t)(1.1 * (double)bytes) + (64u << 20);
}
}  // namespace cd

// ====================================================================== C ABI
namespace cd {
// ---------------------------------------------------------------- serving sessions
// Iteration-level continuous batching on one handle: each of the handle's max_batch slots runs
// the refinement loop of solve_device on its own schedule (outer residual and check; an inner
// FP32 or FP64 PCG solve advanced one chunk of iterations per step; the update), so a slot can
// be given a new right-hand side between two chunks while the others keep iterating.  Every
// kernel is masked per slot and every reduction has a fixed order per slot, so a slot's result
// does not depend on what the other slots do.
enum { SP_FREE = 0, SP_NEW = 1, SP_OUTER = 2, SP_IN32 = 3, SP_IN64 = 4, SP_DONE = 5 };

// refinement-loop state of the masked slots at the start of their solve
__global__ void sess_init_kernel(int B, const int* __restrict__ mask, int* active, int* status,
                                 int* outer, int* inner) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !mask[b]) return;
  active[b] = 1;
  status[b] = CD_NOT_CONVERGED;
  outer[b] = 0;
  inner[b] = 0;
}
// out[b] = sum of the nb partials of solve b, for the masked solves (fixed order)
__global__ void sum_partials_masked_kernel(const double* __restrict__ part, int nb, int B,
                                           double* __restrict__ out, const int* __restrict__ mask) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !mask[b]) return;
  double s = 0.0;
  for (int i = 0; i < nb; ++i) s += part[(size_t)b * nb + i];
  out[b] = s;
}

static cd_status sess_alloc(cd_solver h) {
  const int B = h->Bcap;
  if (!h->s_b.p) {
    if (h->s_b.alloc(8 * (size_t)B * h->N) != cudaSuccess || h->s_x.alloc(8 * (size_t)B * h->N) != cudaSuccess ||
        h->s_mask.alloc(4 * (size_t)B * 4) != cudaSuccess) {
      cudaGetLastError();
      return CD_ENOMEM;
    }
    // no PCG of either state is running
    CD_CUDA_OK(cudaMemsetAsync(h->si[0].p, 0, 4 * (size_t)B, h->s));
    CD_CUDA_OK(cudaMemsetAsync(h->si2[0].p, 0, 4 * (size_t)B, h->s));
    h->sp.assign(B, SP_FREE);
    h->s_alpha.assign(B, 1.0);
    h->s_beta.assign(B, 1.0);
    h->s_t0.resize(B);
    h->h_mask.assign(4 * B, 0);
  }
  return CD_OK;
}

int sess_busy(cd_solver h) {
  std::lock_guard<std::mutex> lk(h->mu);
  int n = 0;
  for (int v : h->sp) n += v != SP_FREE;
  return n;
}

// Takes a free slot for right-hand side b (host, N doubles); it starts at the next step.
cd_status sess_admit(cd_solver h, const double* b_host, double alpha, double beta, int* slot) {
  if (!(alpha > 0) || !(beta > 0) || !std::isfinite(alpha) || !std::isfinite(beta)) return CD_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  cd_status st = sess_alloc(h);
  if (st != CD_OK) return st;
  int k = -1;
  for (int i = 0; i < h->Bcap && k < 0; ++i)
    if (h->sp[i] == SP_FREE) k = i;
  if (k < 0) return CD_ENOMEM;
  CD_CUDA_OK(cudaMemcpyAsync(h->s_b.as<double>() + (size_t)k * h->N, b_host, 8 * (size_t)h->N,
                             cudaMemcpyHostToDevice, h->s));
  h->s_alpha[k] = alpha;
  h->s_beta[k] = beta;
  h->sp[k] = SP_NEW;
  h->s_t0[k] = std::chrono::steady_clock::now();
  *slot = k;
  return CD_OK;
}

// uploads mask j: the slots whose phase is `phase`
static cd_status sess_mask(cd_solver h, int phase, int j) {
  const int B = h->Bcap;
  for (int b = 0; b < B; ++b) h->h_mask[j * B + b] = h->sp[b] == phase;
  CD_CUDA_OK(cudaMemcpyAsync(h->s_mask.as<int>() + j * B, h->h_mask.data() + j * B, 4 * B,
                             cudaMemcpyHostToDevice, h->s));
  return CD_OK;
}

// One step of every occupied slot; `finished` receives the slots whose solve ended.
cd_status sess_step(cd_solver h, std::vector<int>& finished) {
  finished.clear();
  std::lock_guard<std::mutex> lk(h->mu);
  cd_status st = sess_alloc(h);
  if (st != CD_OK) return st;
  const int B = h->Bcap;
  const long long N = h->N;
  const int pc = h->opt.precond;
  const bool ext = h->opt.ext_residual != 0;
  const bool emu = ext && h->opt.emulated_fp64 && h->opt.precision != CD_PREC_FP64;
  double* b = h->s_b.as<double>();
  double* x = h->s_x.as<double>();
  double* xlo = ext ? h->xlo64.as<double>() : nullptr;
  int* mk[4];
  for (int j = 0; j < 4; ++j) mk[j] = h->s_mask.as<int>() + j * B;
  // 1. admissions: parameters (per-solve multigrid data of the new slots), initial state
  std::vector<int> fresh;
  for (int i = 0; i < B; ++i)
    if (h->sp[i] == SP_NEW) fresh.push_back(i);
  if (!fresh.empty()) {
    CD_CUDA_OK(cudaMemcpyAsync(h->alpha.p, h->s_alpha.data(), 8 * B, cudaMemcpyHostToDevice, h->s));
    CD_CUDA_OK(cudaMemcpyAsync(h->beta.p, h->s_beta.data(), 8 * B, cudaMemcpyHostToDevice, h->s));
    h->dev_alpha = h->s_alpha;
    h->dev_beta = h->s_beta;
    for (MgData* mg : {&h->mg, &h->mgD}) {
      const bool used = mg == &h->mg ? (pc == CD_PC_MG || pc == CD_PC_MIM) : (pc == CD_PC_WL && h->have_mgD);
      if (!used) continue;
      if ((st = mg_set_params_slots(*mg, h->d, h->P, h->s_alpha, h->s_beta, fresh, h->s)) != CD_OK)
        return st;
      if ((st = mg_prepare(*mg, B, coef_of(h), h->w64.apply_scratch.as<double>(), h->s)) != CD_OK)
        return st;
    }
    // the batched solver's record of prepared parameters no longer holds
    h->mg_alpha.clear();
    h->mgD_alpha.clear();
    std::vector<int> grp(B);
    CD_CUDA_OK(cudaMemcpyAsync(grp.data(), h->ir_grp.p, 4 * B, cudaMemcpyDeviceToHost, h->s));
    CD_CUDA_OK(cudaStreamSynchronize(h->s));
    for (int i : fresh) {
      const double ratio = std::max(h->s_alpha[i], h->s_beta[i]) / std::min(h->s_alpha[i], h->s_beta[i]);
      grp[i] = (h->opt.precision == CD_PREC_FP32_IR && ratio < h->opt.mixed_switch_ratio) ? 0 : 2;
    }
    CD_CUDA_OK(cudaMemcpyAsync(h->ir_grp.p, grp.data(), 4 * B, cudaMemcpyHostToDevice, h->s));
    if ((st = sess_mask(h, SP_NEW, 0)) != CD_OK) return st;
    sess_init_kernel<<<(B + 127) / 128, 128, 0, h->s>>>(B, mk[0], h->ir_active.as<int>(),
                                                        h->ir_status.as<int>(), h->ir_outer.as<int>(),
                                                        h->ir_inner_total.as<int>());
    count_launch();
    vzero<double>(N, B, x, mk[0], h->s);
    if (ext) vzero<double>(N, B, xlo, mk[0], h->s);
    const int nb = partial_blocks(N);
    launch_dot<double>(b, b, N, B, h->part[1].as<double>(), nb, mk[0], h->s);
    sum_partials_masked_kernel<<<(B + 127) / 128, 128, 0, h->s>>>(h->part[1].as<double>(), nb, B,
                                                                  h->ir_bnorm2.as<double>(), mk[0]);
    count_launch();
    CD_CUDA_OK(cudaStreamSynchronize(h->s));  // grp (host) goes out of scope
    for (int i : fresh) h->sp[i] = SP_OUTER;
  }
  // 2. outer residual and check of the slots due for it; their inner solves start
  if (std::count(h->sp.begin(), h->sp.end(), (int)SP_OUTER)) {
    if ((st = sess_mask(h, SP_OUTER, 0)) != CD_OK) return st;
    int npart = 0;
    if ((st = outer_residual(h, B, b, x, xlo, mk[0], &npart)) != CD_OK) return st;
    ir_check(B, h->part[0].as<double>(), npart, h->ir_bnorm2.as<double>(), h->ir_rnorm.as<double>(),
             h->ir_rrprev.as<double>(), mk[0], h->ir_status.as<int>(), h->ir_relres.as<double>(),
             h->ir_outer.as<int>(), h->ir_grp.as<int>(), h->ir_tol2.as<double>(),
             h->opt.rtol * h->opt.rtol, h->opt.inner_rtol * h->opt.inner_rtol, h->opt.max_outer,
             h->ir_inner_total.as<int>(), h->opt.maxit, emu ? 1e-12 : 1e-30, h->s);
    std::vector<int> still(B), grp(B);
    CD_CUDA_OK(cudaMemcpyAsync(still.data(), mk[0], 4 * B, cudaMemcpyDeviceToHost, h->s));
    CD_CUDA_OK(cudaMemcpyAsync(grp.data(), h->ir_grp.p, 4 * B, cudaMemcpyDeviceToHost, h->s));
    CD_CUDA_OK(cudaStreamSynchronize(h->s));
    // masks 1 / 2: the slots that start an FP32 / FP64 inner solve now
    bool any32 = false, any64 = false;
    for (int i = 0; i < B; ++i) {
      const bool go = h->sp[i] == SP_OUTER && still[i];
      h->h_mask[1 * B + i] = go && grp[i] == 0;
      h->h_mask[2 * B + i] = go && grp[i] != 0;
      any32 |= h->h_mask[1 * B + i] != 0;
      any64 |= h->h_mask[2 * B + i] != 0;
      if (h->sp[i] == SP_OUTER && !still[i]) {
        h->sp[i] = SP_DONE;
        finished.push_back(i);
      }
    }
    CD_CUDA_OK(cudaMemcpyAsync(mk[1], h->h_mask.data() + B, 8 * B, cudaMemcpyHostToDevice, h->s));
    if (any32) {
      ir_cast(N, B, h->r64.as<double>(), h->w32.r.as<float>(), h->ir_rnorm.as<double>(), mk[1], h->s);
      pcg_begin<float>(h, B, pc, mk[1], 0, 1);
    }
    if (any64) {
      scale_div(N, B, h->r64.as<double>(), h->w64.r.as<double>(), h->ir_rnorm.as<double>(), mk[2], h->s);
      set_fp64_emulated(emu ? 1 : 0);
      g_lowp_prec = h->opt.precision == CD_PREC_FP32_IR ? 1 : 0;
      pcg_begin<double>(h, B, pc, mk[2], 1, 1);
      set_fp64_emulated(0);
      g_lowp_prec = 0;
    }
    for (int i = 0; i < B; ++i)
      if (h->sp[i] == SP_OUTER) h->sp[i] = h->h_mask[1 * B + i] ? SP_IN32 : SP_IN64;
  }
  // 3. one chunk of each inner group, then the slots whose inner solve ended take their update
  const bool run32 = std::count(h->sp.begin(), h->sp.end(), (int)SP_IN32) > 0;
  const bool run64 = std::count(h->sp.begin(), h->sp.end(), (int)SP_IN64) > 0;
  const bool fd = pc == CD_PC_FD_D || pc == CD_PC_FD_T;
  const bool mgk = pc == CD_PC_MG || pc == CD_PC_MIM || pc == CD_PC_WL;
  const int flex32 = (mgk || (h->opt.fd_tensor_cores && fd)) ? 1 : 0;
  const int flex64 = (mgk || (h->opt.precision == CD_PREC_FP32_IR && fd)) ? 1 : 0;
  if (run32 &&
      (st = pcg_chunk<float>(h, B, pc, flex32, h->ir_tol2.as<double>(), h->opt.inner_maxit, 0)) != CD_OK)
    return st;
  if (run64) {
    set_fp64_emulated(emu ? 1 : 0);
    g_lowp_prec = h->opt.precision == CD_PREC_FP32_IR ? 1 : 0;
    st = pcg_chunk<double>(h, B, pc, flex64, h->ir_tol2.as<double>(), h->opt.maxit, 1);
    set_fp64_emulated(0);
    g_lowp_prec = 0;
    if (st != CD_OK) return st;
  }
  if (run32 || run64) {
    std::vector<int> a32(B), a64(B);
    CD_CUDA_OK(cudaMemcpyAsync(a32.data(), h->si[0].p, 4 * B, cudaMemcpyDeviceToHost, h->s));
    CD_CUDA_OK(cudaMemcpyAsync(a64.data(), h->si2[0].p, 4 * B, cudaMemcpyDeviceToHost, h->s));
    CD_CUDA_OK(cudaStreamSynchronize(h->s));
    bool e32 = false, e64 = false;
    for (int i = 0; i < B; ++i) {
      h->h_mask[1 * B + i] = h->sp[i] == SP_IN32 && !a32[i];
      h->h_mask[2 * B + i] = h->sp[i] == SP_IN64 && !a64[i];
      e32 |= h->h_mask[1 * B + i] != 0;
      e64 |= h->h_mask[2 * B + i] != 0;
    }
    CD_CUDA_OK(cudaMemcpyAsync(mk[1], h->h_mask.data() + B, 8 * B, cudaMemcpyHostToDevice, h->s));
    if (e32) {
      add_iters_kernel<<<(B + 127) / 128, 128, 0, h->s>>>(B, h->si[1].as<int>(), mk[1],
                                                          h->ir_inner_total.as<int>());
      count_launch();
      if (ext)
        launch_ext_update<float>(N, B, x, xlo, h->w32.x.as<float>(), h->ir_rnorm.as<double>(), mk[1], h->s);
      else
        ir_update(N, B, x, h->w32.x.as<float>(), h->ir_rnorm.as<double>(), mk[1], h->s);
    }
    if (e64) {
      add_iters_kernel<<<(B + 127) / 128, 128, 0, h->s>>>(B, h->si2[1].as<int>(), mk[2],
                                                          h->ir_inner_total.as<int>());
      count_launch();
      if (ext)
        launch_ext_update<double>(N, B, x, xlo, h->w64.x.as<double>(), h->ir_rnorm.as<double>(), mk[2], h->s);
      else
        ir_update64(N, B, x, h->w64.x.as<double>(), h->ir_rnorm.as<double>(), mk[2], h->s);
    }
    for (int i = 0; i < B; ++i)
      if (h->h_mask[1 * B + i] || h->h_mask[2 * B + i]) h->sp[i] = SP_OUTER;
  }
  CD_CUDA_OK(cudaGetLastError());
  return CD_OK;
}

// The result of a finished slot: its solution x (FP64; with the double-FP64 residual the
// rounding of x + x_lo) into x_host, its cd_result (residual of that x); frees the slot.
cd_status sess_take(cd_solver h, int slot, double* x_host, cd_result* res) {
  std::lock_guard<std::mutex> lk(h->mu);
  if (slot < 0 || slot >= (int)h->sp.size() || h->sp[slot] != SP_DONE) return CD_EINVAL;
  const int B = h->Bcap;
  const long long N = h->N;
  for (int i = 0; i < B; ++i) h->h_mask[3 * B + i] = i == slot;
  int* mk3 = h->s_mask.as<int>() + 3 * B;
  CD_CUDA_OK(cudaMemcpyAsync(mk3, h->h_mask.data() + 3 * B, 4 * B, cudaMemcpyHostToDevice, h->s));
  int npart = 0;
  cd_status st = outer_residual(h, B, h->s_b.as<double>(), h->s_x.as<double>(), nullptr, mk3, &npart);
  if (st != CD_OK) return st;
  const int nb = partial_blocks(N);
  launch_dot<double>(h->s_b.as<double>(), h->s_b.as<double>(), N, B, h->part[1].as<double>(), nb, mk3, h->s);
  std::vector<double> prr(npart), pbb(nb);
  int status = 0, outer = 0, inner = 0;
  CD_CUDA_OK(cudaMemcpyAsync(prr.data(), h->part[0].as<double>() + (size_t)slot * npart, 8 * npart,
                             cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaMemcpyAsync(pbb.data(), h->part[1].as<double>() + (size_t)slot * nb, 8 * nb,
                             cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaMemcpyAsync(&status, h->ir_status.as<int>() + slot, 4, cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaMemcpyAsync(&outer, h->ir_outer.as<int>() + slot, 4, cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaMemcpyAsync(&inner, h->ir_inner_total.as<int>() + slot, 4, cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaMemcpyAsync(x_host, h->s_x.as<double>() + (size_t)slot * N, 8 * (size_t)N,
                             cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaStreamSynchronize(h->s));
  double rr = 0, bb = 0;
  for (double v : prr) rr += v;
  for (double v : pbb) bb += v;
  const double rel = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  if (status == CD_OK && !(rel <= h->opt.rtol)) status = CD_NOT_CONVERGED;
  if (res) {
    res->iters_outer = outer;
    res->iters_inner = inner;
    res->relres = rel;
    res->relres_hi = rel;
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - h->s_t0[slot]).count();
    res->status = status;
  }
  h->sp[slot] = SP_FREE;
  return CD_OK;
}
}  // namespace cd

extern "C" {

void cd_default_options(cd_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = CD_PREC_FP32_IR;
  o->precond = CD_PC_FD_D;
  o->maxit = 20000;
  o->rtol = 1e-10;
  o->max_batch = 64;
  o->inner_rtol = 1e-5;
  o->inner_maxit = 4000;
  o->max_outer = 30;
  o->smoother_degree = 2;
  o->mg_m_min = 0;
  o->use_graphs = 1;
  o->chunk = 8;
  o->mixed_switch_ratio = 1e4;
  o->fd_tensor_cores = 1;
  o->autotune = 1;
  o->ext_residual = 1;
  o->emulated_fp64 = 1;
}

size_t cd_dofs(int d, int p, int n) {
  if ((d != 2 && d != 3) || p < 1 || n < 1) return 0;
  size_t m = (size_t)(n + p - 2), r = (size_t)d;
  for (int l = 0; l < d; ++l) r *= m;
  return r;
}

const char* cd_strerror(cd_status s) {
  switch (s) {
    case CD_OK: return "ok";
    case CD_EINVAL: return "invalid argument";
    case CD_ENOMEM: return "out of device memory";
    case CD_ECUDA: return "CUDA error";
    case CD_NOT_CONVERGED: return "not converged";
    case CD_BREAKDOWN: return "Krylov breakdown";
    case CD_TIMEOUT: return "timeout";
    case CD_CANCELLED: return "cancelled";
  }
  return "unknown status";
}

const char* cd_last_error(void) { return cd::last_error(); }
uint64_t cd_kernel_launches(void) { return cd::launches(); }

static cd_status ensure_tband(cd_solver h);
static cd_status ensure_ksmooth(cd_solver h, int kind);

// Per-solve state, Krylov vectors of both precisions and the apply scratch (elements per
// precision); false when an allocation fails.
static bool alloc_workspace(cd_solver h, long long scratch_elems) {
  const int B = h->Bcap;
  const long long N = h->N;
  auto al = [&](DevBuf& bfr, size_t bytes) { return bfr.alloc(bytes) == cudaSuccess; };
  bool ok = al(h->alpha, 8 * B) && al(h->beta, 8 * B);
  for (auto& x : h->sd) ok = ok && al(x, 8 * B);
  for (auto& x : h->si) ok = ok && al(x, 4 * B);
  for (auto& x : h->sd2) ok = ok && al(x, 8 * B);
  for (auto& x : h->si2) ok = ok && al(x, 4 * B);
  for (auto& x : h->part) ok = ok && al(x, 8 * (size_t)B * kMaxPartials);
  ok = ok && al(h->ir_rnorm, 8 * B) && al(h->ir_bnorm2, 8 * B) && al(h->ir_relres, 8 * B) &&
       al(h->ir_active, 4 * B) && al(h->ir_status, 4 * B) && al(h->ir_outer, 4 * B) &&
       al(h->ir_inner_total, 4 * B) && al(h->cnt, 64) && al(h->r64, 8 * (size_t)B * N) &&
       al(h->ir_rrprev, 8 * B) && al(h->ir_grp, 4 * B) && al(h->ir_tol2, 8 * B) &&
       al(h->ir_m0, 4 * B) && al(h->ir_m1, 4 * B) && al(h->ir_m2, 4 * B);
  for (int prec = 0; prec < 2; ++prec) {
    const size_t es = prec == 0 ? 8 : 4;
    Workspace& w = prec == 0 ? h->w64 : h->w32;
    const size_t vb = es * (size_t)B * N;
    ok = ok && al(w.x, vb) && al(w.r, vb) && al(w.z, vb) && al(w.p, vb) && al(w.q, vb) &&
         al(w.fa, vb) && al(w.fb, vb) &&
         al(w.apply_scratch, es * (size_t)std::max<long long>(scratch_elems, 1));
  }
  return ok;
}

cd_status cd_create(cd_solver* out, int d, int p, int n, double alpha, double beta,
                    const cd_options* opt, void* stream) {
  if (!out) return CD_EINVAL;
  *out = nullptr;
  if ((d != 2 && d != 3) || p < 1 || n < 1 || n + p - 2 < 2) {
    set_error("need d in {2,3}, p >= 1, n >= 1, m = n+p-2 >= 2");
    return CD_EINVAL;
  }
  if (!(alpha > 0) || !(beta > 0) || !std::isfinite(alpha) || !std::isfinite(beta)) {
    set_error("alpha and beta must be finite and > 0");
    return CD_EINVAL;
  }
  if (cd_dofs(d, p, n) >= (size_t(1) << 31)) {  // the kernels index one solve's vector in 32 bits
    set_error("d (n+p-2)^d must be below 2^31");
    return CD_EINVAL;
  }
  std::unique_ptr<cd_solver_s> h(new cd_solver_s());
  h->d = d;
  h->p = p;
  h->n = n;
  h->m = n + p - 2;
  h->P = p;
  h->alpha0 = alpha;
  h->beta0 = beta;
  cd_default_options(&h->opt);
  if (opt) h->opt = *opt;
  if (h->opt.max_batch < 1 || h->opt.max_batch > 4096 || h->opt.chunk < 1 || h->opt.maxit < 1 ||
      !(h->opt.rtol > 0) || h->opt.precond < 0 || h->opt.precond > CD_PC_WL || h->opt.precision < 0 ||
      h->opt.precision > 1) {
    set_error("invalid options");
    return CD_EINVAL;
  }
  h->s = static_cast<cudaStream_t>(stream);
  if (prepare_kernels() != 0) {
    set_error(cudaGetErrorString(cudaGetLastError()));
    return CD_ECUDA;
  }
  h->N = (long long)cd_dofs(d, p, n);
  h->Bcap = h->opt.max_batch;
  const int B = h->Bcap;
  const long long N = h->N;
  const int m = h->m, P = h->P, W = 2 * P + 1;
  // 1D bands on every level (finest: quadrature; coarser: Galerkin P^T X P)
  Band M, A, S;
  iga_bands(p, n, P, M, A, S);
  const int m_min = mg_coarsest(d, h->opt.mg_m_min, h->opt.precond);
  for (;;) {
    h->hM.push_back(M);
    h->hA.push_back(A);
    h->hS.push_back(S);
    h->ml.push_back(M.m);
    if (M.m <= m_min || M.m / 2 < 1) break;
    M = coarsen(M);
    A = coarsen(A);
    S = coarsen(S);
  }
  // per level: [3][m][W] row-major bands, [3][W][m] k-major copy, padded to 4 elements
  std::vector<double> all;
  std::vector<std::pair<int, int>> interior;
  std::vector<std::vector<double>> central;
  for (size_t l = 0; l < h->ml.size(); ++l) {
    const int ml = h->ml[l];
    Band* X[3] = {&h->hM[l], &h->hA[l], &h->hS[l]};
    // rows equal to the central row (Toeplitz part) within rounding
    const int ic = ml / 2;
    auto row_ok = [&](int i) {
      for (int x = 0; x < 3; ++x) {
        double mx = 0.0;
        for (double v : X[x]->v) mx = std::max(mx, std::fabs(v));
        for (int k = 0; k < W; ++k) {
          const double a = X[x]->v[(size_t)i * W + k], c = X[x]->v[(size_t)ic * W + k];
          if (std::fabs(a - c) > 1e-14 * mx) return false;
        }
      }
      return true;
    };
    int lo = ic, hi = ic + 1;
    if (ml >= 2 * W + 1) {
      while (lo - 1 >= 0 && row_ok(lo - 1)) --lo;
      while (hi < ml && row_ok(hi)) ++hi;
    } else {
      lo = hi = 0;
    }
    interior.push_back({lo, hi});
    std::vector<double> c(3 * W);
    for (int x = 0; x < 3; ++x)
      for (int k = 0; k < W; ++k) c[x * W + k] = X[x]->v[(size_t)ic * W + k];
    // The central row is made exactly symmetric (M, S) or antisymmetric (A), as the Toeplitz
    // symbols of Section 3.2 are.  The interior rows agree with it up to quadrature rounding;
    // they are replaced by it, so that a kernel reading the constant stencil and one reading the
    // band row see the same coefficients (and produce the same bits).  Then every entry below
    // the diagonal is set from its transpose (the interior row's value where one of the two rows
    // is interior), so M and S stay exactly symmetric and A exactly skew: the operator
    // gamma A (x) A of the kernels is then exactly the printed -alpha A^T (x) A + beta A (x) A^T,
    // and the block matrix exactly symmetric.
    for (int x = 0; x < 3; ++x)
      for (int k = 1; k <= P; ++k) {
        double& up = c[x * W + P + k];
        double& dn = c[x * W + P - k];
        const double v = x == 1 ? 0.5 * (up - dn) : 0.5 * (up + dn);
        up = v;
        dn = x == 1 ? -v : v;
      }
    c[1 * W + P] = 0.0;
    for (int i = lo; i < hi; ++i)
      for (int x = 0; x < 3; ++x)
        for (int k = 0; k < W; ++k) X[x]->v[(size_t)i * W + k] = c[x * W + k];
    for (int x = 0; x < 3; ++x) {
      const double sgn = x == 1 ? -1.0 : 1.0;
      std::vector<double>& v = X[x]->v;
      for (int i = 0; i < ml; ++i)
        for (int k = 1; k <= P && i + k < ml; ++k) {
          const int j = i + k;
          const bool ii = i >= lo && i < hi, jj = j >= lo && j < hi;
          double& upper = v[(size_t)i * W + P + k];  // X(i, j)
          double& lower = v[(size_t)j * W + P - k];  // X(j, i)
          if (!ii && jj)
            upper = sgn * lower;
          else
            lower = sgn * upper;
        }
      if (x == 1)
        for (int i = 0; i < ml; ++i) v[(size_t)i * W + P] = 0.0;
    }
    central.push_back(c);
    h->boff.push_back(all.size());
    for (int x = 0; x < 3; ++x) all.insert(all.end(), X[x]->v.begin(), X[x]->v.end());
    for (int x = 0; x < 3; ++x)
      for (int k = 0; k < W; ++k)
        for (int i = 0; i < ml; ++i) all.push_back(X[x]->v[(size_t)i * W + k]);
    while (all.size() % 4) all.push_back(0.0);
  }
  if (upload(h->bands64, all) != cudaSuccess || upload(h->bands32, cast_vec<float>(all)) != cudaSuccess) {
    set_error("band upload failed");
    return CD_ECUDA;
  }
  for (size_t l = 0; l < h->ml.size(); ++l) {
    register_level(h->bands64.as<double>() + h->boff[l], h->ml[l], P, interior[l].first,
                   interior[l].second, central[l].data());
    if (d == 2) register_level_ff(h->bands64.as<double>() + h->boff[l], h->ml[l], P);
    register_level(h->bands32.as<float>() + h->boff[l], h->ml[l], P, interior[l].first,
                   interior[l].second, central[l].data());
  }
  {
    const char* v = std::getenv("CURLDIV_APPLY_KERNEL");
    const std::string vs = v ? v : "";
    set_apply_variant(vs == "v1" ? 0 : vs == "v2" ? 1 : vs == "v3" ? 3 : 2);
    const char* v64 = std::getenv("CURLDIV_APPLY_KERNEL_FP64");
    const std::string v64s = v64 ? v64 : "";
    set_apply_fp64_variant(v64s == "v3" ? 1 : v64s == "ff" ? 2 : v64s == "ff2" ? 3 : v64s == "ff1" ? 4 : 0);
    const char* v3d = std::getenv("CURLDIV_APPLY3D_KERNEL");
    const std::string v3ds = v3d ? v3d : "";
    set_apply3d_variant(v3ds == "multipass" ? 0 : v3ds == "axis" ? 2 : v3ds == "stream" ? 3
                        : v3ds == "pass64" ? 4 : 1);
    const char* vr = std::getenv("CURLDIV_FF2_ROWS");
    set_ff2_rows(vr ? std::atoi(vr) : 0);
  }
  if (h->opt.precond == CD_PC_FD_D || h->opt.precond == CD_PC_FD_T) {
    cd_status st = ensure_fd(h.get());
    if (st != CD_OK) return st;
  }
  if (h->opt.precond == CD_PC_T_BAND) {
    cd_status st = ensure_tband(h.get());
    if (st != CD_OK) return st;
  }
  // workspace
  const long long scratch3d = (d == 3) ? 21LL * (N / 3) * B : 0;
  if (!alloc_workspace(h.get(), scratch3d)) {
    set_error("workspace allocation failed");
    cudaGetLastError();
    return CD_ENOMEM;
  }
  auto al = [&](DevBuf& bfr, size_t bytes) { return bfr.alloc(bytes) == cudaSuccess; };
  if (h->opt.ext_residual) {  // double-FP64 solution and residual intermediates
    const long long per = ext_scratch_doubles_per_solve(d, m);
    const long long budget = (256LL << 20) / 8;  // doubles of intermediates per launch group
    h->ext_chunk = (int)std::max<long long>(1, std::min<long long>(B, budget / per));
    if (!al(h->xlo64, 8 * (size_t)B * N) || !al(h->ext_scratch, 8 * (size_t)h->ext_chunk * per)) {
      set_error("workspace allocation failed");
      cudaGetLastError();
      return CD_ENOMEM;
    }
  }
  if (cudaMallocHost(&h->h_cnt, 64) != cudaSuccess) return CD_ENOMEM;
  {
    cd_status st = mg_build(h->mg, d, P, h->ml, h->hM, h->hA, h->hS, B,
                            std::max(1, h->opt.smoother_degree), h->bands64.as<double>(),
                            h->bands32.as<float>(), h->boff);
    if (st != CD_OK) return st;
  }
  if (h->opt.precond == CD_PC_MIM || h->opt.precond == CD_PC_WL) {
    cd_status st = ensure_ksmooth(h.get(), h->opt.precond);
    if (st != CD_OK) return st;
  }
  if (h->opt.autotune && d == 3) {  // pick the 3D apply design per level (FP32)
    std::vector<double> ones(B, 1.0);
    if (cudaMemcpyAsync(h->alpha.p, ones.data(), 8 * B, cudaMemcpyHostToDevice, h->s) != cudaSuccess ||
        cudaMemcpyAsync(h->beta.p, ones.data(), 8 * B, cudaMemcpyHostToDevice, h->s) != cudaSuccess) {
      set_error("autotune set-up failed");
      return CD_ECUDA;
    }
    h->dev_alpha = ones;
    h->dev_beta = ones;
    for (size_t l = 0; l < h->ml.size(); ++l)
      tune_apply3d<float>(h->ml[l], P, bands_of<float>(h.get(), l), h->w32.p.as<float>(),
                          h->w32.q.as<float>(), B, coef_of(h.get()),
                          h->w32.apply_scratch.as<float>(), h->s);
  }
  if (h->opt.autotune && d == 2) {  // pick the 2D apply variant per level and precision
    std::vector<double> ones(B, 1.0);
    if (cudaMemcpyAsync(h->alpha.p, ones.data(), 8 * B, cudaMemcpyHostToDevice, h->s) != cudaSuccess ||
        cudaMemcpyAsync(h->beta.p, ones.data(), 8 * B, cudaMemcpyHostToDevice, h->s) != cudaSuccess) {
      set_error("autotune set-up failed");
      return CD_ECUDA;
    }
    h->dev_alpha = ones;
    h->dev_beta = ones;
    for (size_t l = 0; l < h->ml.size(); ++l) {
      tune_apply2d<float>(h->ml[l], P, bands_of<float>(h.get(), l), h->w32.p.as<float>(),
                          h->w32.q.as<float>(), B, coef_of(h.get()), h->s);
      tune_apply2d<double>(h->ml[l], P, bands_of<double>(h.get(), l), h->w64.p.as<double>(),
                           h->w64.q.as<double>(), B, coef_of(h.get()), h->s);
    }
  }
  if (cudaStreamSynchronize(h->s) != cudaSuccess) {
    set_error(cudaGetErrorString(cudaGetLastError()));
    return CD_ECUDA;
  }
  *out = h.release();
  return CD_OK;
}

cd_status cd_create_aniso(cd_solver* out, int d, int p, const int* n, double alpha, double beta,
                          const cd_options* opt, void* stream) {
  if (!out) return CD_EINVAL;
  *out = nullptr;
  if ((d != 2 && d != 3) || p < 1 || !n) {
    set_error("need d in {2,3}, p >= 1 and one interval count per direction");
    return CD_EINVAL;
  }
  long long npc = 1;
  for (int l = 0; l < d; ++l) {
    if (n[l] < 1 || n[l] + p - 2 < 2) {
      set_error("need n_l >= 1 and m_l = n_l+p-2 >= 2 in every direction");
      return CD_EINVAL;
    }
    npc *= n[l] + p - 2;
  }
  if (d * npc >= (1LL << 31)) {
    set_error("d prod_l (n_l+p-2) must be below 2^31");
    return CD_EINVAL;
  }
  if (!(alpha > 0) || !(beta > 0) || !std::isfinite(alpha) || !std::isfinite(beta)) {
    set_error("alpha and beta must be finite and > 0");
    return CD_EINVAL;
  }
  std::unique_ptr<cd_solver_s> h(new cd_solver_s());
  h->aniso = true;
  h->d = d;
  h->p = p;
  h->n = n[0];
  h->P = p;
  for (int l = 0; l < d; ++l) h->ma[l] = n[l] + p - 2;
  h->m = h->ma[0];
  h->alpha0 = alpha;
  h->beta0 = beta;
  cd_default_options(&h->opt);
  h->opt.precond = CD_PC_NONE;
  if (opt) h->opt = *opt;
  if (h->opt.max_batch < 1 || h->opt.max_batch > 4096 || h->opt.chunk < 1 || h->opt.maxit < 1 ||
      !(h->opt.rtol > 0) || h->opt.precision < 0 || h->opt.precision > 1) {
    set_error("invalid options");
    return CD_EINVAL;
  }
  if (h->opt.precond != CD_PC_NONE && h->opt.precond != CD_PC_FD_D) {
    set_error("anisotropic meshes: precond must be CD_PC_NONE or CD_PC_FD_D");
    return CD_EINVAL;
  }
  // the banded passes of the anisotropic apply: FP64 residuals and SIMT FD transforms
  h->opt.ext_residual = 0;
  h->opt.emulated_fp64 = 0;
  h->opt.fd_tensor_cores = 0;
  h->opt.autotune = 0;
  h->s = static_cast<cudaStream_t>(stream);
  if (prepare_kernels() != 0) {
    set_error(cudaGetErrorString(cudaGetLastError()));
    return CD_ECUDA;
  }
  h->N = d * npc;
  h->Bcap = h->opt.max_batch;
  const int P = p, W = 2 * P + 1;
  // 1D bands of every direction ([3][m_l][W] row-major), M and S exactly symmetric, A exactly
  // skew (upper entries copied to the lower ones), as on a uniform mesh
  std::vector<double> all, Uall, Utall, lamall;
  for (int l = 0; l < d; ++l) {
    Band M, A, S;
    iga_bands(p, n[l], P, M, A, S);
    Band* X[3] = {&M, &A, &S};
    const int ml = h->ma[l];
    for (int x = 0; x < 3; ++x) {
      const double sgn = x == 1 ? -1.0 : 1.0;
      std::vector<double>& v = X[x]->v;
      for (int i = 0; i < ml; ++i)
        for (int k = 1; k <= P && i + k < ml; ++k)
          v[(size_t)(i + k) * W + P - k] = sgn * v[(size_t)i * W + P + k];
      if (x == 1)
        for (int i = 0; i < ml; ++i) v[(size_t)i * W + P] = 0.0;
    }
    h->aoff[l] = all.size();
    for (int x = 0; x < 3; ++x) all.insert(all.end(), X[x]->v.begin(), X[x]->v.end());
    while (all.size() % 4) all.push_back(0.0);
    if (h->opt.precond == CD_PC_FD_D) {  // S_l U = M_l U Lambda_l, U^T M_l U = I
      std::vector<double> U, lam;
      if (!gen_eig(ml, band_to_dense(M), band_to_dense(S), U, lam)) {
        set_error("generalized eigen-decomposition failed");
        return CD_EINVAL;
      }
      h->aUoff[l] = Uall.size();
      h->alamoff[l] = lamall.size();
      Uall.insert(Uall.end(), U.begin(), U.end());
      for (int i = 0; i < ml; ++i)
        for (int j = 0; j < ml; ++j) Utall.push_back(U[(size_t)j * ml + i]);
      lamall.insert(lamall.end(), lam.begin(), lam.end());
    }
  }
  for (int l = d; l < 3; ++l) h->aoff[l] = h->aoff[d - 1];
  if (upload(h->bands64, all) != cudaSuccess || upload(h->bands32, cast_vec<float>(all)) != cudaSuccess) {
    set_error("band upload failed");
    return CD_ECUDA;
  }
  if (h->opt.precond == CD_PC_FD_D) {
    for (int l = d; l < 3; ++l) {
      h->aUoff[l] = h->aUoff[d - 1];
      h->alamoff[l] = h->alamoff[d - 1];
    }
    if (upload(h->aU64, Uall) != cudaSuccess || upload(h->aUt64, Utall) != cudaSuccess ||
        upload(h->alam64, lamall) != cudaSuccess || upload(h->aU32, cast_vec<float>(Uall)) != cudaSuccess ||
        upload(h->aUt32, cast_vec<float>(Utall)) != cudaSuccess ||
        upload(h->alam32, cast_vec<float>(lamall)) != cudaSuccess) {
      set_error("eigenbasis upload failed");
      return CD_ECUDA;
    }
  }
  const long long scratch = (long long)(d == 2 ? 6 : 18) * npc * h->Bcap + h->N * h->Bcap;
  if (!alloc_workspace(h.get(), scratch)) {
    set_error("workspace allocation failed");
    cudaGetLastError();
    return CD_ENOMEM;
  }
  if (cudaMallocHost(&h->h_cnt, 64) != cudaSuccess) return CD_ENOMEM;
  if (cudaStreamSynchronize(h->s) != cudaSuccess) {
    set_error(cudaGetErrorString(cudaGetLastError()));
    return CD_ECUDA;
  }
  *out = h.release();
  return CD_OK;
}

cd_status cd_destroy(cd_solver h) {
  if (!h) return CD_EINVAL;
  cudaStreamSynchronize(h->s);
  delete h;
  return CD_OK;
}

static cd_status check_call(cd_solver h, const void* a, const void* b, int nrhs) {
  if (!h || !a || !b) {
    set_error("NULL argument");
    return CD_EINVAL;
  }
  if (nrhs < 1 || nrhs > h->Bcap) {
    set_error("nrhs out of range [1, max_batch]");
    return CD_EINVAL;
  }
  return CD_OK;
}

cd_status cd_apply(cd_solver h, const double* w, double* y, int nrhs, const double* alphas,
                   const double* betas) {
  cd_status st = check_call(h, w, y, nrhs);
  if (st != CD_OK) return st;
  std::lock_guard<std::mutex> lk(h->mu);
  if ((st = set_params(h, nrhs, alphas, betas)) != CD_OK) return st;
  if (apply_level<double>(h, 0, w, y, nullptr, 0, nrhs, nullptr, nullptr, nullptr) != 0) {
    set_error("no apply kernel fits this problem size");
    return CD_EINVAL;
  }
  CD_CUDA_OK(cudaGetLastError());
  return CD_OK;
}

cd_status cd_apply_f32(cd_solver h, const float* w, float* y, int nrhs, const double* alphas,
                       const double* betas) {
  cd_status st = check_call(h, w, y, nrhs);
  if (st != CD_OK) return st;
  std::lock_guard<std::mutex> lk(h->mu);
  if ((st = set_params(h, nrhs, alphas, betas)) != CD_OK) return st;
  if (apply_level<float>(h, 0, w, y, nullptr, 0, nrhs, nullptr, nullptr, nullptr) != 0) {
    set_error("no apply kernel fits this problem size");
    return CD_EINVAL;
  }
  CD_CUDA_OK(cudaGetLastError());
  return CD_OK;
}

cd_status cd_solve(cd_solver h, const double* b, double* x, int nrhs, const double* alphas,
                   const double* betas, cd_result* res) {
  cd_status st = check_call(h, b, x, nrhs);
  if (st != CD_OK) return st;
  std::lock_guard<std::mutex> lk(h->mu);
  std::vector<double> va, vb;
  if ((st = set_params(h, nrhs, alphas, betas, &va, &vb, h->opt.precond)) != CD_OK) return st;
  return solve_device(h, b, x, nullptr, nrhs, res, va, vb);
}

cd_status cd_solve_ext(cd_solver h, const double* b, double* x, double* x_lo, int nrhs,
                       const double* alphas, const double* betas, cd_result* res) {
  cd_status st = check_call(h, b, x, nrhs);
  if (st != CD_OK) return st;
  std::lock_guard<std::mutex> lk(h->mu);
  std::vector<double> va, vb;
  if ((st = set_params(h, nrhs, alphas, betas, &va, &vb, h->opt.precond)) != CD_OK) return st;
  return solve_device(h, b, x, x_lo, nrhs, res, va, vb);
}

cd_status cd_solve_host(cd_solver h, const double* b_host, double* x_host, int nrhs,
                        const double* alphas, const double* betas, cd_result* res) {
  cd_status st = check_call(h, b_host, x_host, nrhs);
  if (st != CD_OK) return st;
  std::lock_guard<std::mutex> lk(h->mu);
  std::vector<double> va, vb;
  if ((st = set_params(h, nrhs, alphas, betas, &va, &vb, h->opt.precond)) != CD_OK) return st;
  const size_t bytes = 8 * (size_t)nrhs * h->N;
  if (!h->b64.p) {
    if (h->b64.alloc(8 * (size_t)h->Bcap * h->N) != cudaSuccess ||
        h->x64.alloc(8 * (size_t)h->Bcap * h->N) != cudaSuccess)
      return CD_ENOMEM;
  }
  CD_CUDA_OK(cudaMemcpyAsync(h->b64.p, b_host, bytes, cudaMemcpyHostToDevice, h->s));
  st = solve_device(h, h->b64.as<double>(), h->x64.as<double>(), nullptr, nrhs, res, va, vb);
  if (st != CD_OK && st != CD_NOT_CONVERGED && st != CD_BREAKDOWN) return st;
  CD_CUDA_OK(cudaMemcpyAsync(x_host, h->x64.p, bytes, cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaStreamSynchronize(h->s));
  return st;
}

// Banded Cholesky factor of T_m(m_{p-1}) (SPD: its eigenvalues lie in [(2/pi)^{2(p-1)}, 1]),
// half-bandwidth q = p - 1, in FP64 on the host; FP64 and FP32 copies on the device.
static cd_status ensure_tband(cd_solver h) {
  if (h->have_tband) return CD_OK;
  if (h->p - 1 > 5) {
    set_error("banded T solve: p <= 6");
    return CD_EINVAL;
  }
  std::vector<double> Lb, dinv;
  if (!tband_factor(h->p, h->m, Lb, dinv)) {
    set_error("banded Cholesky of T failed (not positive definite)");
    return CD_EINVAL;
  }
  if (Lb.empty()) Lb.push_back(0.0);
  if (upload(h->TB64, Lb) != cudaSuccess || upload(h->TBd64, dinv) != cudaSuccess ||
      upload(h->TB32, cast_vec<float>(Lb)) != cudaSuccess ||
      upload(h->TBd32, cast_vec<float>(dinv)) != cudaSuccess) {
    set_error("banded T factor upload failed");
    return CD_ECUDA;
  }
  h->have_tband = true;
  return CD_OK;
}

// The finest-level Krylov post-smoother (p iterations preconditioned by T, banded solves) of
// P_MIM (on the hierarchy of A) or P_WL (on that of D, built here on first use).
static cd_status ensure_ksmooth(cd_solver h, int kind) {
  cd_status st = ensure_tband(h);
  if (st != CD_OK) return st;
  if (kind == CD_PC_WL && !h->have_mgD) {
    st = mg_build(h->mgD, h->d, h->P, h->ml, h->hM, h->hA, h->hS, h->Bcap,
                  std::max(1, h->opt.smoother_degree), h->bands64.as<double>(),
                  h->bands32.as<float>(), h->boff);
    if (st != CD_OK) return st;
    st = mg_set_block_diagonal(h->mgD);
    if (st != CD_OK) return st;
    h->have_mgD = true;
  }
  MgData& mg = kind == CD_PC_WL ? h->mgD : h->mg;
  return mg_setup_ksmooth(mg, h->p, h->TB64.p, h->TBd64.p, h->TB32.p, h->TBd32.p);
}

// ------------------------------------------------------------------ host-only set-up queries
static bool setup_args_ok(int p, int n) {
  if (p < 1 || p > 6 || n < 1 || n + p - 2 < 1) {
    set_error("need 1 <= p <= 6, n >= 1, n + p - 2 >= 1");
    return false;
  }
  return true;
}

cd_status cd_setup_bands(int p, int n, int level, double* M, double* A, double* S, int* m_out,
                         int* P_out) {
  if (!setup_args_ok(p, n) || level < 0) return CD_EINVAL;
  Band Mb, Ab, Sb;
  iga_bands(p, n, p, Mb, Ab, Sb);
  for (int l = 0; l < level; ++l) {
    if (Mb.m / 2 < 1) {
      set_error("cd_setup_bands: level below the coarsest grid");
      return CD_EINVAL;
    }
    Mb = coarsen(Mb);
    Ab = coarsen(Ab);
    Sb = coarsen(Sb);
  }
  if (m_out) *m_out = Mb.m;
  if (P_out) *P_out = Mb.P;
  const size_t bytes = Mb.v.size() * sizeof(double);
  if (M) std::memcpy(M, Mb.v.data(), bytes);
  if (A) std::memcpy(A, Ab.v.data(), bytes);
  if (S) std::memcpy(S, Sb.v.data(), bytes);
  return CD_OK;
}

cd_status cd_setup_eig(int p, int n, int which, double* U, double* lam) {
  if (!setup_args_ok(p, n) || (which != 0 && which != 1)) return CD_EINVAL;
  const int m = n + p - 2;
  std::vector<double> Uv, lv;
  if (which == 0) {
    Band Mb, Ab, Sb;
    iga_bands(p, n, p, Mb, Ab, Sb);
    if (!gen_eig(m, band_to_dense(Mb), band_to_dense(Sb), Uv, lv)) {
      set_error("generalized eigen-decomposition failed");
      return CD_EINVAL;
    }
  } else {
    Band T;
    toeplitz_T_band(p, m, p, T);
    sym_eig(m, band_to_dense(T), Uv, lv);
  }
  if (U) std::memcpy(U, Uv.data(), Uv.size() * sizeof(double));
  if (lam) std::memcpy(lam, lv.data(), lv.size() * sizeof(double));
  return CD_OK;
}

cd_status cd_setup_tband(int p, int n, double* Lb, double* dinv) {
  if (!setup_args_ok(p, n)) return CD_EINVAL;
  std::vector<double> l, dv;
  if (!tband_factor(p, n + p - 2, l, dv)) {
    set_error("banded Cholesky of T failed (not positive definite)");
    return CD_EINVAL;
  }
  if (Lb) std::memcpy(Lb, l.data(), l.size() * sizeof(double));
  if (dinv) std::memcpy(dinv, dv.data(), dv.size() * sizeof(double));
  return CD_OK;
}

cd_status cd_precond(cd_solver h, int kind, const void* r, void* z, int nrhs, const double* alphas,
                     const double* betas, int f32) {
  cd_status st = check_call(h, r, z, nrhs);
  if (st != CD_OK) return st;
  if (kind < CD_PC_NONE || kind > CD_PC_WL) return CD_EINVAL;
  if (h->aniso && kind != CD_PC_NONE && !(kind == CD_PC_FD_D && h->aU64.p)) {
    set_error("anisotropic mesh: only CD_PC_NONE, and CD_PC_FD_D on a handle created with it");
    return CD_EINVAL;
  }
  std::lock_guard<std::mutex> lk(h->mu);
  if (!h->aniso && (kind == CD_PC_FD_D || kind == CD_PC_FD_T)) {
    st = ensure_fd(h);
    if (st != CD_OK) return st;
  }
  if (kind == CD_PC_T_BAND) {
    st = ensure_tband(h);
    if (st != CD_OK) return st;
  }
  if (kind == CD_PC_MIM || kind == CD_PC_WL) {
    st = ensure_ksmooth(h, kind);
    if (st != CD_OK) return st;
  }
  st = set_params(h, nrhs, alphas, betas, nullptr, nullptr, kind);
  if (st != CD_OK) return st;
  if (f32)
    apply_prec<float>(h, kind, nrhs, (const float*)r, (float*)z, nullptr);
  else
    apply_prec<double>(h, kind, nrhs, (const double*)r, (double*)z, nullptr);
  CD_CUDA_OK(cudaGetLastError());
  return CD_OK;
}

int cd_levels(cd_solver h) { return h ? (int)h->ml.size() : 0; }

cd_status cd_symbol_eigs(int d, int p, double alpha, double beta, const double* nu, int mg,
                         double* lam, double* lap, void* stream) {
  if ((d != 2 && d != 3) || p < 1 || p > 8 || mg < 1 || !lam) {
    set_error("cd_symbol_eigs: need d in {2,3}, 1 <= p <= 8, mg >= 1, lam != NULL");
    return CD_EINVAL;
  }
  if (!(alpha > 0) || !(beta > 0) || !std::isfinite(alpha) || !std::isfinite(beta)) {
    set_error("cd_symbol_eigs: alpha and beta must be finite and > 0");
    return CD_EINVAL;
  }
  if (nu)
    for (int l = 0; l < d; ++l)
      if (!(nu[l] > 0) || !std::isfinite(nu[l])) {
        set_error("cd_symbol_eigs: nu must be finite and > 0");
        return CD_EINVAL;
      }
  double np = 1;
  for (int l = 0; l < d; ++l) np *= mg;
  if (np > 4e9) {
    set_error("cd_symbol_eigs: grid too large");
    return CD_EINVAL;
  }
  launch_symbol_eigs(d, p, alpha, beta, nu, mg, lam, lap, static_cast<cudaStream_t>(stream));
  CD_CUDA_OK(cudaGetLastError());
  return CD_OK;
}

struct LanczosCtx {
  cd_solver h;
  int B;
};
static void lanczos_apply(void* ctx, const double* x, double* y) {
  LanczosCtx* c = static_cast<LanczosCtx*>(ctx);
  apply_level<double>(c->h, 0, x, y, nullptr, 0, c->B, nullptr, nullptr, nullptr);
}

cd_status cd_lanczos(cd_solver h, const double* v0, int nrhs, int steps, const double* alphas,
                     const double* betas, double* lam_min, double* lam_max, double* diag,
                     double* offdiag) {
  cd_status st = check_call(h, v0, lam_min ? (const void*)lam_min : (const void*)lam_max, nrhs);
  if (st != CD_OK) return st;
  if (!lam_min || !lam_max || steps < 1 || steps > 4096) {
    set_error("cd_lanczos: need lam_min, lam_max != NULL and 1 <= steps <= 4096");
    return CD_EINVAL;
  }
  std::lock_guard<std::mutex> lk(h->mu);
  if ((st = set_params(h, nrhs, alphas, betas)) != CD_OK) return st;
  const size_t need = 8 * (size_t)h->Bcap * steps;
  if (h->lz_a.bytes < need) {
    if (h->lz_a.alloc(need) != cudaSuccess || h->lz_b.alloc(need) != cudaSuccess) {
      cudaGetLastError();
      set_error("cd_lanczos: allocation failed");
      return CD_ENOMEM;
    }
  }
  const int B = nrhs;
  CD_CUDA_OK(cudaMemsetAsync(h->lz_a.p, 0, need, h->s));
  CD_CUDA_OK(cudaMemsetAsync(h->lz_b.p, 0, need, h->s));
  LanczosCtx ctx{h, B};
  lanczos_run(h->N, B, steps, v0, h->w64.x.as<double>(), h->w64.r.as<double>(),
              h->w64.z.as<double>(), h->lz_a.as<double>(), h->lz_b.as<double>(),
              h->sd[0].as<double>(), h->sd[1].as<double>(), h->si[0].as<int>(),
              h->si[1].as<int>(), h->part[0].as<double>(), lanczos_apply, &ctx, h->s);
  std::vector<double> a((size_t)B * steps), b((size_t)B * steps);
  std::vector<int> used(B);
  CD_CUDA_OK(cudaMemcpyAsync(a.data(), h->lz_a.p, a.size() * 8, cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaMemcpyAsync(b.data(), h->lz_b.p, b.size() * 8, cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaMemcpyAsync(used.data(), h->si[1].p, B * 4, cudaMemcpyDeviceToHost, h->s));
  CD_CUDA_OK(cudaStreamSynchronize(h->s));
  for (int i = 0; i < B; ++i) {
    const int k = std::max(1, std::min(steps, used[i]));
    tridiag_extremes(&a[(size_t)i * steps], &b[(size_t)i * steps], k, &lam_min[i], &lam_max[i]);
  }
  if (diag) std::memcpy(diag, a.data(), a.size() * 8);
  if (offdiag) std::memcpy(offdiag, b.data(), b.size() * 8);
  return CD_OK;
}

cd_status cd_get_bands(cd_solver h, int level, double* M, double* A, double* S, int* m_out,
                       int* P_out) {
  if (!h || level < 0 || level >= (int)h->ml.size()) return CD_EINVAL;
  if (m_out) *m_out = h->ml[level];
  if (P_out) *P_out = h->P;
  const size_t n = h->hM[level].v.size();
  if (M) std::memcpy(M, h->hM[level].v.data(), n * 8);
  if (A) std::memcpy(A, h->hA[level].v.data(), n * 8);
  if (S) std::memcpy(S, h->hS[level].v.data(), n * 8);
  return CD_OK;
}

cd_status cd_get_eig(cd_solver h, int which, double* U, double* lam) {
  if (!h || h->aniso || (which != 0 && which != 1)) return CD_EINVAL;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    cd_status st = ensure_fd(h);
    if (st != CD_OK) return st;
  }
  const std::vector<double>& Us = which == 0 ? h->UD : h->UT;
  const std::vector<double>& ls = which == 0 ? h->lamD : h->lamT;
  if (U) std::memcpy(U, Us.data(), Us.size() * 8);
  if (lam) std::memcpy(lam, ls.data(), ls.size() * 8);
  return CD_OK;
}

cd_status cd_restrict(cd_solver h, int level, const double* fine, double* coarse, int nrhs) {
  cd_status st = check_call(h, fine, coarse, nrhs);
  if (st != CD_OK) return st;
  if (level < 0 || level + 1 >= (int)h->ml.size()) return CD_EINVAL;
  mg_restrict<double>(h->d, h->ml[level], h->ml[level + 1], nrhs, fine, coarse, nullptr, h->s);
  CD_CUDA_OK(cudaGetLastError());
  return CD_OK;
}

cd_status cd_prolong(cd_solver h, int level, const double* coarse, double* fine, int nrhs) {
  cd_status st = check_call(h, coarse, fine, nrhs);
  if (st != CD_OK) return st;
  if (level < 0 || level + 1 >= (int)h->ml.size()) return CD_EINVAL;
  mg_prolong_add<double>(h->d, h->ml[level], h->ml[level + 1], nrhs, coarse, fine, nullptr, h->s);
  CD_CUDA_OK(cudaGetLastError());
  return CD_OK;
}

}  // extern "C"
