// Fast-diagonalisation contractions on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// C[z](r, c) = sum_k A[z](r, k) B[z](k, c) for one axis of the FD transform (see
// launch_fd_axis): FP32 operands read as TF32 by tcgen05.mma kind::tf32, FP32 accumulation in
// tensor memory.  One CTA (4 warps) owns a 128 x 128 output tile; K (= m) is consumed in
// chunks of 32 staged into shared memory in the canonical K-major layout without swizzle
// (8-row x 16-byte core matrices; leading-byte offset = next core matrix along K, stride-byte
// offset = next 8-row group), double-buffered.  Thread 0 issues the MMAs and commits them to an
// mbarrier; the epilogue reads the accumulator with tcgen05.ld and applies the FD eigenvalue
// scaling.  The tensors' rows are m floats long (m odd for most (p, n)), which TMA's 16-byte
// stride rule excludes, so the CTA stages its tiles itself (coalesced global loads).
// Every mbarrier wait is bounded; on expiry the kernel raises *err and skips its stores.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "krylov.h"

namespace cd {

namespace {
constexpr int TM = 128, TN = 128, KC = 32;                  // tile and K chunk
constexpr int A_BYTES = TM * KC * 4, B_BYTES = TN * KC * 4;  // 16 KB each
constexpr uint32_t kWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, k) inside a [rows x KC] K-major no-swizzle chunk.
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)(((row >> 3) * (KC / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
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

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

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

template <typename T>
__global__ void __launch_bounds__(128, 1) fd_tc_kernel(int Mr, int Nc, int K, const float* __restrict__ A,
                                                       long long ars, long long acs, long long abs_,
                                                       const float* __restrict__ Bm, long long brs,
                                                       long long bcs, long long bbs, float* __restrict__ C,
                                                       long long crs, long long ccs, long long cbs,
                                                       FdScale<float> sc, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_base_sh;
  const int z = blockIdx.z;
  const int r0 = blockIdx.y * TM, c0 = blockIdx.x * TN;
  const float* Az = A + (long long)z * abs_;
  const float* Bz = Bm + (long long)z * bbs;
  const int tid = threadIdx.x, warp = tid >> 5;
  unsigned char* bufA[2] = {smem, smem + A_BYTES + B_BYTES};
  unsigned char* bufB[2] = {smem + A_BYTES, smem + 2 * A_BYTES + B_BYTES};

  if (warp == 0) {  // tensor-memory allocation: 128 FP32 columns = the 128 x 128 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
                     smem_u32(&tmem_base_sh)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;

  const int nchunks = (K + KC - 1) / KC;
  uint32_t phase[2] = {0, 0};
  bool ok = true;
  for (int ch = 0; ch < nchunks; ++ch) {
    const int buf = ch & 1;
    // the MMAs that read this buffer two chunks ago must be complete before it is rewritten
    if (ch >= 2) {
      if (!mbar_wait(&bars[buf], phase[buf])) ok = false;
      phase[buf] ^= 1;
    }
    const int k0 = ch * KC;
    // stage A chunk [TM x KC] and B chunk [TN x KC] (as (row = c, k)) in the core layout
    if (acs == 1) {  // lanes cover one 8-row x 4-float core block: conflict-free stores
      for (int e = tid; e < TM * KC; e += 128) {
        const int blk = e >> 5, kk = (blk % (KC / 4)) * 4 + (e & 3);
        const int rr = (blk / (KC / 4)) * 8 + ((e >> 2) & 7);
        const int gr = r0 + rr, gk = k0 + kk;
        const float v = (gr < Mr && gk < K) ? Az[gr * ars + gk] : 0.f;
        *reinterpret_cast<float*>(bufA[buf] + core_off(rr, kk)) = v;
      }
    } else {
      for (int e = tid; e < TM * KC; e += 128) {
        const int rr = e % TM, kk = e / TM;
        const int gr = r0 + rr, gk = k0 + kk;
        const float v = (gr < Mr && gk < K) ? Az[gr * ars + gk * acs] : 0.f;
        *reinterpret_cast<float*>(bufA[buf] + core_off(rr, kk)) = v;
      }
    }
    if (bcs == 1) {
      for (int e = tid; e < TN * KC; e += 128) {
        const int cc = e % TN, kk = e / TN;
        const int gc = c0 + cc, gk = k0 + kk;
        const float v = (gc < Nc && gk < K) ? Bz[gk * brs + gc] : 0.f;
        *reinterpret_cast<float*>(bufB[buf] + core_off(cc, kk)) = v;
      }
    } else {
      for (int e = tid; e < TN * KC; e += 128) {
        const int cc = e / KC, kk = e % KC;
        const int gc = c0 + cc, gk = k0 + kk;
        const float v = (gc < Nc && gk < K) ? Bz[gk * brs + gc * bcs] : 0.f;
        *reinterpret_cast<float*>(bufB[buf] + core_off(cc, kk)) = v;
      }
    }
    // generic-proxy writes -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(bufA[buf]), b0 = smem_u32(bufB[buf]);
#pragma unroll
      for (int s = 0; s < KC / 8; ++s) {  // K = 8 per MMA = two 16-byte core matrices
        const uint64_t ad = smem_desc(a0 + s * 256), bd = smem_desc(b0 + s * 256);
        const uint32_t acc = (ch > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&bars[buf])));
    }
  }
  // wait for the last commit of each buffer in use
  {
    const int lastbuf = (nchunks - 1) & 1;
    if (!mbar_wait(&bars[lastbuf], phase[lastbuf])) ok = false;
    if (nchunks >= 2) {
      const int other = lastbuf ^ 1;
      if (!mbar_wait(&bars[other], phase[other])) ok = false;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  // epilogue: warp w reads accumulator lanes 32w..32w+31 (one output row per thread)
  const int row = r0 + warp * 32 + (tid & 31);
  float* Cz = C + (long long)z * cbs;
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
  }
#pragma unroll 1
  for (int cb = 0; cb < TN; cb += 8) {
    uint32_t v[8];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    if (ok && row < Mr) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = c0 + cb + j;
        if (col >= Nc) continue;
        float out = __uint_as_float(v[j]);
        float* dst = Cz + (long long)row * crs + (long long)col * ccs;
        if (sc.mode) {
          long long off = dst - sc.base;
          const long long bc = off / sc.per;
          long long rem = off - bc * sc.per;
          const int bsol = (int)(bc / sc.d), comp = (int)(bc % sc.d);
          double den = sc.mode == 1 ? 0.0 : 1.0;
          for (int l = sc.d - 1; l >= 0; --l) {
            const int kl = (int)(rem % sc.m);
            rem /= sc.m;
            const double lam = (double)sc.lam[kl];
            if (sc.mode == 1)
              den += (l == comp ? sc.beta[bsol] : sc.alpha[bsol]) * lam;
            else
              den *= lam;
          }
          out = (float)((double)out / den);
        }
        *dst = out;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
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
  const size_t smem = 2 * (A_BYTES + B_BYTES);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(fd_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  if (I == 1) {
    const long long R = O;
    const long long rows_per_z = 65535LL * TM;
    for (long long rlo = 0; rlo < R; rlo += rows_per_z) {
      const int Rz = (int)std::min(rows_per_z, R - rlo);
      dim3 grid((m + TN - 1) / TN, (Rz + TM - 1) / TM, 1);
      fd_tc_kernel<float><<<grid, 128, smem, s>>>(Rz, m, m, in + rlo * m, m, 1, 0, G, m, 1, 0,
                                                  out + rlo * m, m, 1, 0, sc, g_tc_err);
      count_launch();
    }
  } else {
    const long long zmax = 65535;
    for (long long o0 = 0; o0 < O; o0 += zmax) {
      const int nz = (int)std::min(zmax, O - o0);
      dim3 grid((unsigned)((I + TN - 1) / TN), (m + TM - 1) / TM, nz);
      fd_tc_kernel<float><<<grid, 128, smem, s>>>(m, (int)I, m, G, 1, m, 0, in + o0 * m * I, I, 1,
                                                  (long long)m * I, out + o0 * m * I, I, 1,
                                                  (long long)m * I, sc, g_tc_err);
      count_launch();
    }
  }
  return true;
}

int fd_tc_error() {
  if (!g_tc_err) return 0;
  int h = 0;
  cudaMemcpy(&h, g_tc_err, sizeof(int), cudaMemcpyDeviceToHost);
  return h;
}

}  // namespace cd
