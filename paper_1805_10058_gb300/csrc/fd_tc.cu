// Fast-diagonalisation contractions on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One axis of the FD transform (see launch_fd_axis) as C(R, n) = sum_k A(R, k) B(n, k):
// R runs over the accumulator's rows (tensor-memory lanes), n over the eigen index along the
// axis (the MMA's N, a multiple of 16 up to 256 chosen per launch so that m is covered with
// little padding), k over the contraction (= m).  FP32 operands are read as TF32 by
// tcgen05.mma kind::tf32, with FP32 accumulation in tensor memory.  One CTA (4 warps) owns 128
// rows and one N tile; K is consumed in chunks of 32 staged into shared memory in the canonical
// K-major layout without swizzle (8-row x 16-byte core matrices; leading-byte offset = next core
// matrix along K, stride-byte offset = next 8-row group), double-buffered.  Thread 0 issues the
// MMAs and commits them to an mbarrier; the epilogue reads the accumulator with tcgen05.ld and
// applies the FD eigenvalue scaling.  The tensors' rows are m floats long (m odd for most
// (p, n)), which TMA's 16-byte stride rule excludes, so the CTA stages its tiles itself: a warp
// fills one 128-byte core matrix per step (conflict-free shared stores), its lanes ordered along
// whichever operand index is contiguous in global memory.
//
// Orientation: for an axis other than the last, R = (block, position along the later axes),
// the unit-stride index of the output, so a warp's stores are contiguous; blocks are merged
// into one row range so that tiles do not restart per block.  For the last axis R is the data
// row and the output's unit stride is n: the epilogue transposes through shared memory.
// Every mbarrier wait is bounded; on expiry the kernel raises *err and skips its stores.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "krylov.h"

namespace cd {

namespace {
constexpr int TM = 128, KC = 32, TN_MAX = 144, NST = 3;  // row tile, K chunk, N cap, stages
constexpr int NW = 8, NTHR = 32 * NW;                    // warps, threads per CTA
constexpr int A_BYTES = TM * KC * 4;                     // 16 KB
constexpr int EPI_BYTES = NW * 32 * 65 * 4;              // transposing epilogue, per CTA
constexpr int MAX_SMEM = NST * (A_BYTES + TN_MAX * KC * 4);  // 102 KB at N = 144
constexpr uint32_t kWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 4-byte asynchronous global -> shared copy; zero-filled when !valid (src is not read)
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  const uint64_t lbo = 128, sbo = (KC / 4) * 128;
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(lbo >> 4) << 16;
  d |= (uint64_t)(sbo >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of tcgen05
  return d;                // base offset 0, no swizzle
}

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = tn
__device__ __forceinline__ uint32_t idesc_tf32(int tn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(tn >> 3) << 17) |
         ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
// bounded wait for the phase `parity` of an mbarrier; false when the limit expires
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
}  // namespace

// C(R, n) = sum_k A(R, k) B(n, k); row R = z * Ia + c (block z, position c).
struct FdTcArgs {
  int M, N, K, TN, Ia;
  long long a_zs, a_rs, a_ks;  // A(R, k) at A[z * a_zs + c * a_rs + k * a_ks]
  long long b_ns, b_ks;        // B(n, k) at B[n * b_ns + k * b_ks]
  long long c_zs, c_rs, c_ns;  // C(R, n) at C[z * c_zs + c * c_rs + n * c_ns]
  const float* A;
  const float* B;
  float* C;
};

__global__ void __launch_bounds__(NTHR, 1) fd_tc_kernel(FdTcArgs g, FdScale<float> sc,
                                                        int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[NST];
  __shared__ uint32_t tmem_base_sh;
  const int r0 = blockIdx.x * TM, c0 = blockIdx.y * g.TN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {  // tensor-memory allocation: 256 FP32 columns (the N tile is <= 144)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
                     smem_u32(&tmem_base_sh)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < NST; ++i) mbar_init(&bars[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;

  // staging roles, fixed over K: this thread's rows of A (2 of the 16 row groups) and of B (up
  // to 3 of at most 18), each with its source pointer at k = its lane's k offset
  const int rowsA = (min(TM, g.M - r0) + 7) & ~7, rowsB = (min(g.TN, g.N - c0) + 7) & ~7;
  const bool a_kfast = g.a_ks == 1, b_kfast = g.b_ks == 1;
  const int a_r8 = a_kfast ? (lane >> 2) : (lane & 7), a_k4 = a_kfast ? (lane & 3) : (lane >> 3);
  const int b_r8 = b_kfast ? (lane >> 2) : (lane & 7), b_k4 = b_kfast ? (lane & 3) : (lane >> 3);
  const float* pA[2];
  bool aok[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int R = r0 + (warp + NW * i) * 8 + a_r8;
    aok[i] = R < g.M;
    const int z = aok[i] ? R / g.Ia : 0;
    pA[i] = aok[i] ? g.A + (long long)z * g.a_zs + (long long)(R - z * g.Ia) * g.a_rs +
                         (long long)a_k4 * g.a_ks
                   : g.A;
  }
  const float* pB[3];
  bool bok[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int n = c0 + (warp + NW * i) * 8 + b_r8;
    bok[i] = n < g.N;
    pB[i] = bok[i] ? g.B + (long long)n * g.b_ns + (long long)b_k4 * g.b_ks : g.B;
  }

  const int nchunks = (g.K + KC - 1) / KC;
  const uint32_t idesc = idesc_tf32(g.TN);
  const int stage_bytes = A_BYTES + g.TN * KC * 4;
  const uint32_t smem0 = smem_u32(smem);
  // Issues this thread's copies of K chunk ch into stage st (rows past the matrix edge are not
  // staged: they only feed accumulator rows / columns that are never stored; the K tail is
  // zero-filled).
  auto issue_rows = [&](const float* p0, bool rok, long long ks, uint32_t dst, int k0, int k4) {
    if (k0 + KC <= g.K) {
      const long long step = rok ? 4 * ks : 0;
      const float* p = rok ? p0 + (long long)k0 * ks : p0;
#pragma unroll
      for (int kb = 0; kb < KC / 4; ++kb) {
        cp_async4(dst + kb * 128, p, rok);
        p += step;
      }
    } else {
#pragma unroll
      for (int kb = 0; kb < KC / 4; ++kb) {
        const bool v = rok && k0 + kb * 4 + k4 < g.K;
        cp_async4(dst + kb * 128, v ? p0 + (long long)(k0 + kb * 4) * ks : p0, v);
      }
    }
  };
  auto issue_chunk = [&](int ch, int st) {
    const int k0 = ch * KC;
    const uint32_t sA = smem0 + st * stage_bytes, sB = sA + A_BYTES;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int rb = warp + NW * i;
      if (rb * 8 >= rowsA) break;
      issue_rows(pA[i], aok[i], g.a_ks, sA + rb * (KC / 4) * 128 + a_r8 * 16 + a_k4 * 4, k0, a_k4);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int rb = warp + NW * i;
      if (rb * 8 >= rowsB) break;
      issue_rows(pB[i], bok[i], g.b_ks, sB + rb * (KC / 4) * 128 + b_r8 * 16 + b_k4 * 4, k0, b_k4);
    }
  };
  bool ok = true;
#pragma unroll
  for (int c = 0; c < NST - 1; ++c) {
    if (c < nchunks) issue_chunk(c, c);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int ch = 0; ch < nchunks; ++ch) {
    const int st = ch % NST;
    // refill the stage of chunk ch - 1 with chunk ch + NST - 1 once its MMAs have completed
    const int nxt = ch + NST - 1;
    if (nxt < nchunks) {
      const int sn = nxt % NST;
      if (nxt >= NST && !mbar_wait(&bars[sn], ((nxt - NST) / NST) & 1)) ok = false;
      issue_chunk(nxt, sn);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NST - 1) : "memory");  // chunk ch landed
    // generic-proxy writes -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem0 + st * stage_bytes, b0 = a0 + A_BYTES;
#pragma unroll
      for (int s = 0; s < KC / 8; ++s) {  // K = 8 per MMA = two 16-byte core matrices
        const uint64_t ad = smem_desc(a0 + s * 256), bd = smem_desc(b0 + s * 256);
        const uint32_t acc = (ch > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&bars[st])));
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  // the last commit tracks every MMA issued before it
  if (!mbar_wait(&bars[(nchunks - 1) % NST], ((nchunks - 1) / NST) & 1)) ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!ok && tid == 0) atomicExch(err, 1);
  const int ncol = min(g.TN, g.N - c0);
  // two warps per 32-lane quarter of the accumulator (a warp may read only its own quarter,
  // warp % 4); they split the columns
  const int quarter = warp & 3, half = warp >> 2;
  const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16);
  if (g.c_rs == 1) {
    // direct: this thread's row R is the output's unit-stride index
    const int R = r0 + quarter * 32 + lane;
    const bool rok = R < g.M;
    const int z = rok ? R / g.Ia : 0, c = rok ? R - z * g.Ia : 0;
    float* crow = g.C + (long long)z * g.c_zs + c;
    // FD scaling (forward pass along axis 0): the row is the flat index of axes 1..d-1 inside
    // block z = (solve, component), the columns the axis-0 eigen index; the row's part of the
    // eigenvalue sum (FD-D) or product (FD-T) is formed once.
    double srow = 0.0, coef0 = 1.0;
    if (sc.mode && rok) {
      const int bsol = z / sc.d, comp = z - bsol * sc.d;
      int rem = c;
      srow = sc.mode == 1 ? 0.0 : 1.0;
      for (int l = sc.d - 1; l >= 1; --l) {
        const int kl = rem % sc.m;
        rem /= sc.m;
        const double lam = (double)sc.lam[kl];
        if (sc.mode == 1)
          srow += (l == comp ? sc.beta[bsol] : sc.alpha[bsol]) * lam;
        else
          srow *= lam;
      }
      if (sc.mode == 1) coef0 = comp == 0 ? sc.beta[bsol] : sc.alpha[bsol];
    }
    // the transform is TF32: the per-element step of the scaling is FP32 (the row's part, a
    // sum of up to d - 1 products, was formed in FP64)
    const float srowf = (float)srow, coef0f = (float)coef0;
#pragma unroll 1
    for (int cb = 8 * half; cb < ncol; cb += 16) {
      uint32_t v[8];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7])
          : "r"(tbase + (uint32_t)cb));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (ok && rok) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (cb + j >= ncol) break;
          const int n = c0 + cb + j;
          float out = __uint_as_float(v[j]);
          if (sc.mode) {
            const float lam0 = sc.lam[n];
            out = __fdividef(out, sc.mode == 1 ? fmaf(coef0f, lam0, srowf) : srowf * lam0);
          }
          crow[(long long)n * g.c_ns] = out;
        }
      }
    }
  } else {
    // transposed through shared memory (the staging buffers are free now): a warp moves 32 rows
    // x 64 columns at a time and stores each row's columns contiguously
    __syncthreads();
    float* sm = reinterpret_cast<float*>(smem) + warp * (32 * 65);
#pragma unroll 1
    for (int cb0 = 64 * half; cb0 < ncol; cb0 += 128) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        uint32_t v[8];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7])
            : "r"(tbase + (uint32_t)(cb0 + 8 * q)));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int j = 0; j < 8; ++j) sm[lane * 65 + 8 * q + j] = __uint_as_float(v[j]);
      }
      __syncwarp();
      if (ok) {
        for (int rr = 0; rr < 32; ++rr) {
          const int R = r0 + quarter * 32 + rr;
          if (R >= g.M) break;
          const int z = g.Ia == INT_MAX ? 0 : R / g.Ia, c = R - z * g.Ia;
          float* crow = g.C + (long long)z * g.c_zs + (long long)c * g.c_rs;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int cc = cb0 + lane + 32 * h;
            if (cc < ncol) crow[(long long)(c0 + cc) * g.c_ns] = sm[rr * 65 + lane + 32 * h];
          }
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  }
}

static int* g_tc_err = nullptr;

// Same contraction as launch_fd_axis<float>, on tcgen05.  Returns false when unavailable.
bool launch_fd_axis_tc(int d, int m, int axis, int B, const float* G, const float* in, float* out,
                       FdScale<float> sc, cudaStream_t s) {
  if (!g_tc_err) {
    if (cudaMalloc(&g_tc_err, sizeof(int)) != cudaSuccess) return false;
    cudaMemset(g_tc_err, 0, sizeof(int));
  }
  long long I = 1;
  for (int l = axis + 1; l < d; ++l) I *= m;
  long long O = (long long)B * d;
  for (int l = 0; l < axis; ++l) O *= m;
  if (sc.mode && I == 1) return false;  // the scaling epilogue expects an axis before the last
  if (O * I > INT_MAX) return false;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(fd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
    attr = true;
  }
  // N tile: cover m with as few tiles of at most 144 as possible, each a multiple of 16 (at
  // 144, three stages of operands take 102 KB: two CTAs per SM)
  const int nt = (m + 143) / 144;
  const int tn = std::max(16, ((m + nt - 1) / nt + 15) / 16 * 16);
  FdTcArgs g{};
  g.N = m;
  g.K = m;
  g.TN = tn;
  g.B = G;  // G[k * m + n]: the eigen index n of the output at unit stride
  g.b_ns = 1;
  g.b_ks = m;
  if (I == 1) {
    // last axis: out[r][n] = sum_k in[r][k] G[k][n], rows R = data rows
    g.M = (int)O;
    g.Ia = INT_MAX;
    g.A = in;
    g.a_zs = 0;
    g.a_rs = m;
    g.a_ks = 1;
    g.C = out;
    g.c_zs = 0;
    g.c_rs = m;
    g.c_ns = 1;
  } else {
    // out[o][n][c] = sum_k G[k][n] in[o][k][c], rows R = (o, c), c at unit stride
    g.M = (int)(O * I);
    g.Ia = (int)I;
    g.A = in;
    g.a_zs = (long long)m * I;
    g.a_rs = 1;
    g.a_ks = I;
    g.C = out;
    g.c_zs = (long long)m * I;
    g.c_rs = 1;
    g.c_ns = I;
  }
  const size_t smem = std::max((size_t)NST * (A_BYTES + tn * KC * 4), (size_t)EPI_BYTES);
  dim3 grid((unsigned)((g.M + TM - 1) / TM), (unsigned)((m + tn - 1) / tn), 1);
  fd_tc_kernel<<<grid, NTHR, smem, s>>>(g, sc, g_tc_err);
  count_launch();
  return true;
}

int fd_tc_error() {
  if (!g_tc_err) return 0;
  int h = 0;
  cudaMemcpy(&h, g_tc_err, sizeof(int), cudaMemcpyDeviceToHost);
  return h;
}

}  // namespace cd
