// surrogate.cu -- kernels of the crack-map surrogate (a U-Net that maps a
// notched-plate run's inputs to its cracked-element map; see
// include/cem_surrogate.h).
//
// Activations are BF16 in NHWC layout, accumulation is FP32, weights are
// kept in FP32 (master copy, Adam state) and mirrored in BF16 for the
// tensor-core GEMMs.  The 3x3 convolution is an implicit GEMM
//   y[p, n] = sum_k A[p, k] W[n, k],  p = pixel, k = (ky, kx, c)
// whose A rows are gathered from the input on the fly (zero outside the
// image) with 16-byte cp.async copies into a 3-stage shared-memory ring,
// fed to mma.sync m16n8k16 BF16 through ldmatrix.  The data gradient is the
// same kernel applied to the output gradient with the weights transposed and
// flipped (written by the Adam kernel); the weight gradient is a second
// implicit GEMM over pixels, split along the pixels into fixed chunks whose
// FP32 partial sums are added in chunk order (deterministic).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cem_surrogate.h"

namespace {

typedef uint16_t bf16_t;  // BF16 storage

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float bf2f(bf16_t v) { return __uint_as_float((uint32_t)v << 16); }
__device__ __forceinline__ bf16_t f2bf(float f) {
  __nv_bfloat16 h = __float2bfloat16_rn(f);
  return *reinterpret_cast<bf16_t *>(&h);
}

// ------------------------------------------------------------ conv 3x3
constexpr int FBM = 128, FBN = 64, FBK = 32, FST = 3, FPAD = FBK + 8;

struct ConvArgs {
  const bf16_t *x;   // [P, ldx] input pixels (channels 0..Cin-1 used)
  const bf16_t *w;   // [N, K] weights, K = 9 * Cin, k = (ky * 3 + kx) * Cin + c
  const float *bias; // [N] or null
  bf16_t *y;         // [P, ldy] output, channels yoff .. yoff + N - 1
  const bf16_t *mask;  // [P, ldm] or null: outputs where mask <= 0 are set to 0
  int B, H, W, Cin, ldx, N, K, relu, ldy, yoff, P, ldm;
};

__global__ void __launch_bounds__(256) k_conv3x3(ConvArgs a) {
  __shared__ __align__(128) bf16_t As[FST][FBM][FPAD];
  __shared__ __align__(128) bf16_t Bs[FST][FBN][FPAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int p0 = blockIdx.x * FBM, n0 = blockIdx.y * FBN;
  const int HW = a.H * a.W, cpt = a.Cin >> 3;
  const int KT = (a.K + FBK - 1) / FBK;
  // this thread's two A rows and its 8-wide k chunk
  const int kc = tid & 3;
  int rb[2], rh[2], rw[2];
  bool rok[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int p = p0 + (tid >> 2) + r * 64;
    rok[r] = p < a.P;
    const int pp = rok[r] ? p : 0;
    rb[r] = pp / HW;
    const int rem = pp - rb[r] * HW;
    rh[r] = rem / a.W;
    rw[r] = rem - rh[r] * a.W;
  }
  auto load_tile = [&](int kt, int s) {
    const int q = kt * (FBK / 8) + kc;  // 8-wide chunk of k
    const int tap = q / cpt, c0 = (q - tap * cpt) * 8;
    const int ky = tap / 3, kx = tap - ky * 3;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int hh = rh[r] + ky - 1, ww = rw[r] + kx - 1;
      const bool ok = rok[r] && tap < 9 && hh >= 0 && hh < a.H && ww >= 0 && ww < a.W;
      const bf16_t *src = ok ? a.x + ((size_t)(rb[r] * a.H + hh) * a.W + ww) * a.ldx + c0 : a.x;
      cp_async16(&As[s][(tid >> 2) + r * 64][kc * 8], src, ok ? 16 : 0);
    }
    const int n = n0 + (tid >> 2), k = kt * FBK + kc * 8;
    const bool okb = n < a.N && k < a.K;
    const bf16_t *srcb = okb ? a.w + (size_t)n * a.K + k : a.w;
    cp_async16(&Bs[s][tid >> 2][kc * 8], srcb, okb ? 16 : 0);
  };

  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

#pragma unroll
  for (int s = 0; s < FST - 1; ++s) {
    if (s < KT) load_tile(s, s);
    cp_async_commit();
  }
  for (int kt = 0; kt < KT; ++kt) {
    cp_async_wait<FST - 2>();
    __syncthreads();
    const int nk = kt + FST - 1;
    if (nk < KT) load_tile(nk, nk % FST);
    cp_async_commit();
    const int s = kt % FST;
#pragma unroll
    for (int kk = 0; kk < FBK; kk += 16) {
      uint32_t af[2][4], bfr[2][4];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
        ldsm_x4(af[mi], &As[s][wm * 32 + mi * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
      for (int nj = 0; nj < 2; ++nj) {
        const int mat = lane >> 3, r = lane & 7;
        ldsm_x4(bfr[nj], &Bs[s][wn * 32 + nj * 16 + (mat >> 1) * 8 + r][kk + (mat & 1) * 8]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
          mma_bf16(acc[mi][ni], af[mi], bfr[ni >> 1][(ni & 1) * 2], bfr[ni >> 1][(ni & 1) * 2 + 1]);
    }
  }
  cp_async_wait<0>();
  // epilogue: bias, ReLU, BF16 pairs
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
      const int n = n0 + wn * 32 + ni * 8 + (lane & 3) * 2;
      if (n >= a.N) continue;
      const float b0 = a.bias ? a.bias[n] : 0.f, b1 = a.bias ? a.bias[n + 1] : 0.f;
#pragma unroll
      for (int hr = 0; hr < 2; ++hr) {
        const int p = p0 + wm * 32 + mi * 16 + (lane >> 2) + hr * 8;
        if (p >= a.P) continue;
        float v0 = acc[mi][ni][hr * 2] + b0, v1 = acc[mi][ni][hr * 2 + 1] + b1;
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (a.mask) {
          const uint32_t mk = *reinterpret_cast<const uint32_t *>(a.mask + (size_t)p * a.ldm + n);
          if (!(bf2f((bf16_t)(mk & 0xffff)) > 0.f)) v0 = 0.f;
          if (!(bf2f((bf16_t)(mk >> 16)) > 0.f)) v1 = 0.f;
        }
        const uint32_t pk = (uint32_t)f2bf(v0) | ((uint32_t)f2bf(v1) << 16);
        *reinterpret_cast<uint32_t *>(a.y + (size_t)p * a.ldy + a.yoff + n) = pk;
      }
    }
}

// ------------------------------------------------ conv 3x3 on tcgen05
// The same implicit GEMM on the 5th-generation tensor cores: a CTA of four
// warps owns 128 pixels x BN channels; K advances 64 at a time (one 128-byte
// swizzle atom of BF16).  Operands are gathered with 16-byte cp.async copies
// straight into the K-major 128-byte-swizzled layout the MMA descriptors
// describe (row r of a tile at r * 128 bytes, its 16-byte chunk c at
// chunk position c ^ (r & 7)), in a 2-stage ring: one stage is copied
// while the MMAs read the other, and the small ring lets two to five CTAs
// share an SM (by BN), which hides the gathers better than a deeper ring
// (4 stages: 29.7 ms per training step, 3: 23.5 ms, 2: 21.3 ms).  One thread issues
// tcgen05.mma (M = 128, N = BN, K = 16 each) into a TMEM accumulator of BN
// FP32 columns; tcgen05.commit arrives on the stage's mbarrier when the MMAs
// reading it are done, which frees the stage for the next copies.  The
// epilogue reads TMEM with tcgen05.ld (warp w: rows 32w .. 32w+31).  Every
// mbarrier wait is bounded; a wait that gives up records a timeout
// (cem_sg_timeouts), and the CTA stops issuing work, waits (bounded) for the
// MMAs already issued, and frees its TMEM only once they are done.
constexpr int TCM = 128, TCK = 64, TCS = 2;
constexpr long TC_SPIN = 1L << 24;  // mbarrier polls (with a short sleep) before a wait gives up

__device__ int g_tc_timeouts;  // waits that gave up (device-wide, cumulative)

__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
// true when the barrier's phase with the given parity has completed
// (non-blocking test)
__device__ __forceinline__ bool mbar_test(uint64_t *bar, int parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity));
  return ok != 0;
}
// bounded wait: about a second at most, then false
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, int parity) {
  for (long i = 0; i < TC_SPIN; ++i) {
    if (mbar_test(bar, parity)) return true;
    if (i > 64) __nanosleep(32);
  }
  return false;
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);       // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}

// instruction descriptor: D FP32, A and B BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int BN>
struct TcSmem {
  uint8_t A[TCS][TCM * 128];
  uint8_t B[TCS][BN * 128];
  uint64_t mma_bar[TCS];
  uint32_t tmem;
  int fail;
};
// the epilogue stages a 128 x (BN + 8) BF16 tile over the operand ring
static_assert(TCM * (32 + 8) * 2 <= TCS * TCM * 128 + TCS * 32 * 128, "staging");
static_assert(TCM * (256 + 8) * 2 <= TCS * TCM * 128 + TCS * 256 * 128, "staging");

template <int BN>
__global__ void __launch_bounds__(128, 1) k_conv3x3_tc(ConvArgs a) {
  extern __shared__ uint8_t tc_raw[];
  TcSmem<BN> &T = *reinterpret_cast<TcSmem<BN> *>(
      (reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int p0 = blockIdx.x * TCM, n0 = blockIdx.y * BN;
  const int HW = a.H * a.W, cpt = a.Cin >> 3;
  const int KB = (a.K + TCK - 1) / TCK;
  const int c = tid & 7;  // this thread's 16-byte chunk column in every tile row

  if (tid == 0) {
    for (int s = 0; s < TCS; ++s) mbar_init(&T.mma_bar[s], 1);
    T.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&T.tmem)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = T.tmem;

  // rows of A this thread copies: (tid >> 3) + 16 i, i < 8
  int rh[8], rw[8], rb[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int p = p0 + (tid >> 3) + 16 * i;
    if (p < a.P) {
      rb[i] = p / HW;
      const int rem = p - rb[i] * HW;
      rh[i] = rem / a.W;
      rw[i] = rem - rh[i] * a.W;
    } else {
      rb[i] = -1; rh[i] = 0; rw[i] = 0;
    }
  }
  auto load_stage = [&](int kb, int s) {
    const int q = kb * (TCK / 8) + c;  // 8-wide k chunk
    const int tap = q / cpt, c0 = (q - tap * cpt) * 8;
    const int ky = tap / 3, kx = tap - ky * 3;
    const uint32_t abase = smem_u32(T.A[s]), bbase = smem_u32(T.B[s]);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = (tid >> 3) + 16 * i;
      const int hh = rh[i] + ky - 1, ww = rw[i] + kx - 1;
      const bool ok = rb[i] >= 0 && tap < 9 && hh >= 0 && hh < a.H && ww >= 0 && ww < a.W;
      const bf16_t *src = ok ? a.x + ((size_t)(rb[i] * a.H + hh) * a.W + ww) * a.ldx + c0 : a.x;
      const uint32_t dst = abase + row * 128 + ((c ^ (row & 7)) << 4);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                   "r"(ok ? 16 : 0));
    }
    const int k = kb * TCK + c * 8;
#pragma unroll
    for (int i = 0; i < BN / 16; ++i) {
      const int row = (tid >> 3) + 16 * i;
      const int n = n0 + row;
      const bool ok = n < a.N && k < a.K;
      const bf16_t *src = ok ? a.w + (size_t)n * a.K + k : a.w;
      const uint32_t dst = bbase + row * 128 + ((c ^ (row & 7)) << 4);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                   "r"(ok ? 16 : 0));
    }
  };

  constexpr uint32_t idesc = tc_idesc(TCM, BN);
  bool failed = false;
  int last_kb = -1;  // the last stage whose MMAs were issued
#pragma unroll
  for (int s = 0; s < TCS - 1; ++s) {
    if (s < KB) load_stage(s, s);
    cp_async_commit();
  }
  for (int kb = 0; kb < KB && !failed; ++kb) {
    const int s = kb % TCS;
    cp_async_wait<TCS - 2>();
    asm volatile("fence.proxy.async.shared::cta;\n" ::);
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      const uint64_t ad = sw128_desc(smem_u32(T.A[s])), bd = sw128_desc(smem_u32(T.B[s]));
#pragma unroll
      for (int k = 0; k < TCK / 16; ++k) {
        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
        // +32 bytes (encoded +2) per K = 16 slice inside the swizzle atom
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad + 2 * k), "l"(bd + 2 * k), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(&T.mma_bar[s])));
    }
    last_kb = kb;
    const int nk = kb + TCS - 1;
    if (nk < KB) {
      if (kb >= 1 && !mbar_wait(&T.mma_bar[(kb - 1) % TCS], ((kb - 1) / TCS) & 1)) {
        failed = true;
        T.fail = 1;
      }
      if (!failed) load_stage(nk, nk % TCS);
    }
    cp_async_commit();
    failed = __syncthreads_or(failed) != 0;
  }
  cp_async_wait<0>();
  // all MMAs done: the last commit tracks every earlier one
  if (!failed && !mbar_wait(&T.mma_bar[(KB - 1) % TCS], ((KB - 1) / TCS) & 1)) failed = true;
  failed = __syncthreads_or(failed) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);

  if (!failed) {
    // TMEM -> (bias, ReLU) -> BF16 tile in shared memory (the operand ring is
    // free now), then coalesced 16-byte stores with the mask applied
    constexpr int LDS = BN + 8;  // padded row of the staged tile (bf16)
    bf16_t *stile = reinterpret_cast<bf16_t *>(T.A[0]);
    const int m = warp * 32 + lane;  // TMEM lane = tile row
#pragma unroll 1
    for (int cb = 0; cb < BN; cb += 32) {
      uint32_t r[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
            "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
            "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
            "=r"(r[31])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        const int n = n0 + cb + j;
        float v0 = __uint_as_float(r[j]), v1 = __uint_as_float(r[j + 1]);
        if (a.bias && n < a.N) {
          v0 += a.bias[n];
          v1 += a.bias[n + 1];
        }
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        *reinterpret_cast<uint32_t *>(stile + m * LDS + cb + j) =
            (uint32_t)f2bf(v0) | ((uint32_t)f2bf(v1) << 16);
      }
    }
    __syncthreads();
    const bool vec = (a.N & 7) == 0 && (a.ldy & 7) == 0 && (a.yoff & 7) == 0 &&
                     (!a.mask || (a.ldm & 7) == 0);
    for (int idx = tid; idx < TCM * (BN / 8); idx += 128) {
      const int row = idx / (BN / 8), ch = (idx - row * (BN / 8)) * 8;
      const int p = p0 + row, n = n0 + ch;
      if (p >= a.P || n >= a.N) continue;
      uint4 v = *reinterpret_cast<const uint4 *>(stile + row * LDS + ch);
      if (vec) {
        if (a.mask) {
          const uint4 mk = *reinterpret_cast<const uint4 *>(a.mask + (size_t)p * a.ldm + n);
          uint32_t *vw = reinterpret_cast<uint32_t *>(&v);
          const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (!(bf2f((bf16_t)(mw[q] & 0xffff)) > 0.f)) vw[q] &= 0xffff0000u;
            if (!(bf2f((bf16_t)(mw[q] >> 16)) > 0.f)) vw[q] &= 0x0000ffffu;
          }
        }
        *reinterpret_cast<uint4 *>(a.y + (size_t)p * a.ldy + a.yoff + n) = v;
      } else {
        const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
        for (int q = 0; q < 4 && n + 2 * q < a.N; ++q) {
          uint32_t w2 = vw[q];
          if (a.mask) {
            const uint32_t mk =
                *reinterpret_cast<const uint32_t *>(a.mask + (size_t)p * a.ldm + n + 2 * q);
            if (!(bf2f((bf16_t)(mk & 0xffff)) > 0.f)) w2 &= 0xffff0000u;
            if (!(bf2f((bf16_t)(mk >> 16)) > 0.f)) w2 &= 0x0000ffffu;
          }
          *reinterpret_cast<uint32_t *>(a.y + (size_t)p * a.ldy + a.yoff + n + 2 * q) = w2;
        }
      }
    }
  } else if (tid == 0) {
    atomicAdd(&g_tc_timeouts, 1);
  }
  // After a wait gave up, MMAs may still be in flight: wait (bounded) for the
  // last issued commit, which tracks every earlier MMA, before the TMEM is
  // freed; if that wait gives up too, the CTA exits without freeing it (the
  // results of the call are invalid in either case; cem_sg_timeouts says so).
  bool drained = true;
  if (failed && last_kb >= 0)
    drained = __syncthreads_and(mbar_wait(&T.mma_bar[last_kb % TCS], (last_kb / TCS) & 1)) != 0;
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (warp == 0 && drained)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(BN));
}

template <int BN>
size_t tc_smem_bytes() {
  return sizeof(TcSmem<BN>) + 1024;
}

template <int BN>
cudaError_t launch_conv_tc(const ConvArgs &a, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc<BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc_smem_bytes<BN>());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((a.P + TCM - 1) / TCM, (a.N + BN - 1) / BN);
  k_conv3x3_tc<BN><<<grid, 128, tc_smem_bytes<BN>(), st>>>(a);
  return cudaGetLastError();
}

int g_use_tc = 1;  // cem_sg_set_gemm_path

// ---------------------------------------------------- conv 3x3 weight grad
// dW[n, k] = sum_p dY[p, n] * A[p, k] over the pixels of split z, written
// to ws[z][n][k]; k = (ky * 3 + kx) * Cin + c as in the forward weights.
constexpr int GBM = 64, GBN = 64, GBK = 32, GST = 3, GPAD = 64 + 8;

struct WgradArgs {
  const bf16_t *x;   // [P, ldx] forward input
  const bf16_t *dy;  // [P, lddy] output gradient (channels 0..N-1)
  float *ws;         // [splits][N][K]
  float *wsb;        // [splits][N] bias partials (null: no bias gradient)
  int B, H, W, Cin, ldx, lddy, N, K, P, chunk;  // chunk: pixels per split
};

__global__ void __launch_bounds__(256) k_conv3x3_wgrad(WgradArgs a) {
  __shared__ __align__(128) bf16_t As[GST][GBK][GPAD];  // [pixel][n]
  __shared__ __align__(128) bf16_t Bs[GST][GBK][GPAD];  // [pixel][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps, each 32 (n) x 16 (k)
  const int m0 = blockIdx.x * GBM, k0 = blockIdx.y * GBN, z = blockIdx.z;
  const int pbeg = z * a.chunk, pend = min(a.P, pbeg + a.chunk);
  const int HW = a.H * a.W, cpt = a.Cin >> 3;
  const int KT = (pend - pbeg + GBK - 1) / GBK;
  const int prow = tid >> 3, ch = tid & 7;
  // this thread's k chunk is fixed: tap and channel
  const int kq = (k0 >> 3) + ch;
  const int tap = kq / cpt, c0 = (kq - tap * cpt) * 8;
  const int ky = tap / 3, kx = tap - ky * 3;
  const bool kok = k0 + ch * 8 < a.K;
  const bool nok = m0 + ch * 8 < a.N;
  auto load_tile = [&](int kt, int s) {
    const int p = pbeg + kt * GBK + prow;
    const bool pok = p < pend;
    const bf16_t *srca = (pok && nok) ? a.dy + (size_t)p * a.lddy + m0 + ch * 8 : a.dy;
    cp_async16(&As[s][prow][ch * 8], srca, (pok && nok) ? 16 : 0);
    bool ok = pok && kok;
    const bf16_t *srcb = a.x;
    if (ok) {
      const int b = p / HW, rem = p - b * HW, h = rem / a.W, w = rem - h * a.W;
      const int hh = h + ky - 1, ww = w + kx - 1;
      ok = hh >= 0 && hh < a.H && ww >= 0 && ww < a.W;
      if (ok) srcb = a.x + ((size_t)(b * a.H + hh) * a.W + ww) * a.ldx + c0;
    }
    cp_async16(&Bs[s][prow][ch * 8], srcb, ok ? 16 : 0);
  };
  float acc[2][2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  // bias: the k-tile-0 blocks also sum dY over their pixels, channel
  // n = tid & 63 over pixel rows (tid >> 6) + 4 r of each staged tile
  const bool do_bias = a.wsb && blockIdx.y == 0;
  float bsum = 0.f;
#pragma unroll
  for (int s = 0; s < GST - 1; ++s) {
    if (s < KT) load_tile(s, s);
    cp_async_commit();
  }
  for (int kt = 0; kt < KT; ++kt) {
    cp_async_wait<GST - 2>();
    __syncthreads();
    const int nk = kt + GST - 1;
    if (nk < KT) load_tile(nk, nk % GST);
    cp_async_commit();
    const int s = kt % GST;
    if (do_bias) {
#pragma unroll
      for (int r = 0; r < GBK / 4; ++r) bsum += bf2f(As[s][(tid >> 6) + 4 * r][tid & 63]);
    }
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 16) {
      const int mat = lane >> 3, r = lane & 7;
      uint32_t af[2][4], bq[4];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
        ldsm_x4_t(af[mi], &As[s][kk + (mat >> 1) * 8 + r][wm * 32 + mi * 16 + (mat & 1) * 8]);
      ldsm_x4_t(bq, &Bs[s][kk + (mat & 1) * 8 + r][wn * 16 + (mat >> 1) * 8]);
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        mma_bf16(acc[mi][0], af[mi], bq[0], bq[1]);
        mma_bf16(acc[mi][1], af[mi], bq[2], bq[3]);
      }
    }
  }
  cp_async_wait<0>();
  if (do_bias) {
    __shared__ float red[4][64];
    red[tid >> 6][tid & 63] = bsum;
    __syncthreads();
    if (tid < 64 && m0 + tid < a.N)
      a.wsb[(size_t)z * a.N + m0 + tid] = (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
  }
  float *out = a.ws + (size_t)z * a.N * a.K;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 2; ++ni) {
      const int k = k0 + wn * 16 + ni * 8 + (lane & 3) * 2;
      if (k >= a.K) continue;
#pragma unroll
      for (int hr = 0; hr < 2; ++hr) {
        const int n = m0 + wm * 32 + mi * 16 + (lane >> 2) + hr * 8;
        if (n >= a.N) continue;
        *reinterpret_cast<float2 *>(out + (size_t)n * a.K + k) =
            make_float2(acc[mi][ni][hr * 2], acc[mi][ni][hr * 2 + 1]);
      }
    }
}

// out[i] = sum_z ws[z][i] in z order
__global__ void k_reduce_splits(const float *ws, int splits, long n, float *out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += ws[(size_t)z * n + i];
    out[i] = s;
  }
}


// ------------------------------------------- weight gradient on tcgen05
// dW^T[k'][o] = sum_p A[p][k'] dY[p][o] with k' = (ky * 3 + kx) * Cin + c and
// A the shifted input (zero outside the image): M = k' (128 per CTA), N = o
// (BN), K = pixels, split into fixed pixel chunks (grid z) whose FP32 tiles
// go to a workspace and are added in chunk order.  Both operands are read in
// their natural NHWC layout, i.e. MN-major for the MMA: in shared memory
// each pixel is a 128-byte row of 64 k' (or o) values, 8 pixels form a
// 1024-byte swizzle atom (16-byte chunk c of row r at c ^ (r & 7)), atoms
// along K are 1024 bytes apart (SBO) and 64-wide atoms along M or N are
// 8192 bytes apart (LBO).  One thread issues the MMAs (K = 16 = two atoms
// each), tcgen05.commit frees the stage, the epilogue writes the transposed
// tile (coalesced along k') with tcgen05.ld.
constexpr int WTM = 128, WTK = 64;

// MN-major, 128-byte swizzle
__device__ __forceinline__ uint64_t mn_desc(uint32_t saddr, uint32_t lbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__host__ __device__ constexpr uint32_t tc_idesc_mn(int M, int N) {
  return tc_idesc(M, N) | (1u << 15) | (1u << 16);
}

template <int BN>
struct TwSmem {
  uint8_t A[TCS][WTM * WTK * 2];  // 16 KB: 2 atoms along k' of 64 pixels x 128 B
  uint8_t B[TCS][BN * WTK * 2];   // BN / 64 atoms along o
  uint64_t mma_bar[TCS];
  uint32_t tmem;
};

template <int BN>
__global__ void __launch_bounds__(128, 1) k_conv3x3_wgrad_tc(WgradArgs a) {
  extern __shared__ uint8_t tw_raw[];
  TwSmem<BN> &T = *reinterpret_cast<TwSmem<BN> *>(
      (reinterpret_cast<uintptr_t>(tw_raw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * WTM, n0 = blockIdx.y * BN, z = blockIdx.z;
  const int pbeg = z * a.chunk, pend = min(a.P, pbeg + a.chunk);
  const int KB = (pend - pbeg + WTK - 1) / WTK;
  const int HW = a.H * a.W;

  if (tid == 0) {
    for (int s = 0; s < TCS; ++s) mbar_init(&T.mma_bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&T.tmem)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = T.tmem;

  // A: this thread's k' chunk (8 values) is fixed; its pixel rows are
  // (tid >> 4) + 8 i of each stage
  const int ck = tid & 15;
  const int kq = m0 + ck * 8;
  const bool kok = kq < a.K;
  const int tap = kok ? kq / a.Cin : 0, c0 = kok ? kq - tap * a.Cin : 0;
  const int ky = tap / 3, kx = tap - ky * 3;
  const uint32_t aoff_c = (uint32_t)((ck >> 3) * 8192);
  // (b, h, w) of this thread's first pixel row, advanced by 8 pixels per
  // row and 64 per stage without divisions (W >= 8 keeps each carry single)
  int pb0, ph0, pw0;
  {
    const int p = pbeg + (tid >> 4);
    pb0 = p / HW;
    const int rem = p - pb0 * HW;
    ph0 = rem / a.W;
    pw0 = rem - ph0 * a.W;
  }
  auto advance = [&](int &b, int &h, int &w, int n) {
    w += n;
    while (w >= a.W) {
      w -= a.W;
      if (++h == a.H) { h = 0; ++b; }
    }
  };
  auto load_stage = [&](int kb, int s) {
    const int pst = pbeg + kb * WTK;
    const uint32_t abase = smem_u32(T.A[s]), bbase = smem_u32(T.B[s]);
    int b = pb0, h = ph0, w = pw0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int pr = (tid >> 4) + 8 * i;
      const int p = pst + pr;
      bool ok = kok && p < pend;
      const bf16_t *src = a.x;
      if (ok) {
        const int hh = h + ky - 1, ww = w + kx - 1;
        ok = hh >= 0 && hh < a.H && ww >= 0 && ww < a.W;
        if (ok) src = a.x + ((size_t)(b * a.H + hh) * a.W + ww) * a.ldx + c0;
      }
      if (i < 7) advance(b, h, w, 8);
      const int g = pr >> 3, r = pr & 7;
      const uint32_t dst = abase + aoff_c + g * 1024 + r * 128 + (((ck & 7) ^ r) << 4);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                   "r"(ok ? 16 : 0));
    }
    advance(pb0, ph0, pw0, WTK);  // stages are loaded in increasing order
    constexpr int CPR = BN / 8;            // 16-byte chunks per pixel row
    constexpr int RPP = 128 / CPR;         // pixel rows per pass
#pragma unroll
    for (int i = 0; i < WTK / RPP; ++i) {
      const int pr = tid / CPR + RPP * i, cc = tid % CPR;
      const int p = pst + pr, n = n0 + cc * 8;
      const bool ok = p < pend && n < a.N;
      const bf16_t *src = ok ? a.dy + (size_t)p * a.lddy + n : a.dy;
      const int g = pr >> 3, r = pr & 7;
      const uint32_t dst = bbase + (cc >> 3) * 8192 + g * 1024 + r * 128 + (((cc & 7) ^ r) << 4);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                   "r"(ok ? 16 : 0));
    }
  };

  constexpr uint32_t idesc = tc_idesc_mn(WTM, BN);
  bool failed = false;
  int last_kb = -1;  // the last stage whose MMAs were issued
#pragma unroll
  for (int s = 0; s < TCS - 1; ++s) {
    if (s < KB) load_stage(s, s);
    cp_async_commit();
  }
  for (int kb = 0; kb < KB && !failed; ++kb) {
    const int s = kb % TCS;
    cp_async_wait<TCS - 2>();
    asm volatile("fence.proxy.async.shared::cta;\n" ::);
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      const uint32_t as = smem_u32(T.A[s]), bs = smem_u32(T.B[s]);
#pragma unroll
      for (int k = 0; k < WTK / 16; ++k) {
        // B: with a single 64-wide atom along o the atom stride is unused
        const uint64_t ad = mn_desc(as + k * 2048, 8192),
                       bd = mn_desc(bs + k * 2048, BN > 64 ? 8192 : 1024);
        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(&T.mma_bar[s])));
    }
    last_kb = kb;
    const int nk = kb + TCS - 1;
    if (nk < KB) {
      if (kb >= 1 && !mbar_wait(&T.mma_bar[(kb - 1) % TCS], ((kb - 1) / TCS) & 1)) failed = true;
      if (!failed) load_stage(nk, nk % TCS);
    }
    cp_async_commit();
    failed = __syncthreads_or(failed) != 0;
  }
  cp_async_wait<0>();
  if (!failed && KB > 0 && !mbar_wait(&T.mma_bar[(KB - 1) % TCS], ((KB - 1) / TCS) & 1))
    failed = true;
  failed = __syncthreads_or(failed) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);

  float *out = a.ws + (size_t)z * a.N * a.K;
  const int kr = m0 + warp * 32 + lane;  // this lane's k' row of the tile
  if (!failed) {
#pragma unroll 1
    for (int cb = 0; cb < BN; cb += 32) {
      uint32_t r[32];
      if (KB > 0) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
            "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
              "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
              "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
              "=r"(r[31])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) r[j] = 0u;
      }
      if (kr < a.K) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + cb + j;
          if (n < a.N) out[(size_t)n * a.K + kr] = __uint_as_float(r[j]);
        }
      }
    }
  } else if (tid == 0) {
    atomicAdd(&g_tc_timeouts, 1);
  }
  // After a wait gave up, MMAs may still be in flight: wait (bounded) for the
  // last issued commit, which tracks every earlier MMA, before the TMEM is
  // freed; if that wait gives up too, the CTA exits without freeing it (the
  // results of the call are invalid in either case; cem_sg_timeouts says so).
  bool drained = true;
  if (failed && last_kb >= 0)
    drained = __syncthreads_and(mbar_wait(&T.mma_bar[last_kb % TCS], (last_kb / TCS) & 1)) != 0;
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (warp == 0 && drained)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(BN));
}

// per-channel sums of dY [P, ld] (channels 0..C-1, C a multiple of 8) over
// fixed pixel chunks: ws[chunk][C]; 16-byte loads, a fixed reduction order
__global__ void __launch_bounds__(256) k_colsum8(const bf16_t *t, int P, int C, int ld,
                                                 int chunk, float *ws) {
  __shared__ float red[256][9];
  const int C8 = C >> 3;
  const int lanes = 256 / C8;  // pixel lanes per block (C <= 2048)
  const int cg = threadIdx.x % C8, pl = threadIdx.x / C8;
  const int z = blockIdx.x;
  const int pend = min(P, (z + 1) * chunk);
  float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (pl < lanes) {
    for (int p = z * chunk + pl; p < pend; p += lanes) {
      const uint4 v = *reinterpret_cast<const uint4 *>(t + (size_t)p * ld + cg * 8);
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        s[2 * q] += bf2f((bf16_t)(w[q] & 0xffff));
        s[2 * q + 1] += bf2f((bf16_t)(w[q] >> 16));
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) red[threadIdx.x][q] = s[q];
  __syncthreads();
  if (threadIdx.x < C8) {
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int l = 0; l < lanes; ++l)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] += red[l * C8 + threadIdx.x][q];
#pragma unroll
    for (int q = 0; q < 8; ++q) ws[(size_t)z * C + threadIdx.x * 8 + q] = acc[q];
  }
}

template <int BN>
size_t tw_smem_bytes() {
  return sizeof(TwSmem<BN>) + 1024;
}

template <int BN>
cudaError_t launch_wgrad_tc(const WgradArgs &a, int splits, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_wgrad_tc<BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tw_smem_bytes<BN>());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((a.K + WTM - 1) / WTM, (a.N + BN - 1) / BN, splits);
  k_conv3x3_wgrad_tc<BN><<<grid, 128, tw_smem_bytes<BN>(), st>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------- elementwise
// dy[p, c] = 0 where y[p, c] <= 0 (gradient through ReLU, given its output)
__global__ void k_relu_bwd(bf16_t *dy, int lddy, const bf16_t *y, int ldy, long P, int C) {
  const long n = P * C;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long p = i / C;
    const int c = (int)(i - p * C);
    if (!(bf2f(y[p * ldy + c]) > 0.f)) dy[p * lddy + c] = 0;
  }
}

// Pooling and upsampling move 8 channels (16 bytes) per thread; channel
// counts, strides and offsets are multiples of 8.
__device__ __forceinline__ void unpack8(uint4 v, float f[8]) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    f[2 * q] = bf2f((bf16_t)(w[q] & 0xffff));
    f[2 * q + 1] = bf2f((bf16_t)(w[q] >> 16));
  }
}
__device__ __forceinline__ uint4 pack8(const float f[8]) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) w[q] = (uint32_t)f2bf(f[2 * q]) | ((uint32_t)f2bf(f[2 * q + 1]) << 16);
  return make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ uint4 ld8(const bf16_t *p) { return *reinterpret_cast<const uint4 *>(p); }
__device__ __forceinline__ void st8(bf16_t *p, uint4 v) { *reinterpret_cast<uint4 *>(p) = v; }

// 2x2 max pooling: x [B, 2H, 2W] (pixel stride ldx) -> y [B, H, W, C] dense
__global__ void k_maxpool2(const bf16_t *x, int ldx, int B, int H, int W, int C, bf16_t *y) {
  const int C8 = C >> 3;
  const long n = (long)B * H * W * C8;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C8) * 8;
    const long pix = i / C8;
    const int w = (int)(pix % W), h = (int)((pix / W) % H), b = (int)(pix / ((long)W * H));
    const size_t base = ((size_t)(b * 2 * H + 2 * h) * (2 * W) + 2 * w) * ldx + c;
    const size_t row = (size_t)2 * W * ldx;
    float v[4][8], o[8];
    unpack8(ld8(x + base), v[0]);
    unpack8(ld8(x + base + ldx), v[1]);
    unpack8(ld8(x + base + row), v[2]);
    unpack8(ld8(x + base + row + ldx), v[3]);
#pragma unroll
    for (int q = 0; q < 8; ++q) o[q] = fmaxf(fmaxf(v[0][q], v[1][q]), fmaxf(v[2][q], v[3][q]));
    st8(y + (size_t)pix * C + c, pack8(o));
  }
}

// gradient of 2x2 max pooling to the first maximum of each window, plus an
// optional skip gradient (dskip [.., ldskip] at channel offset skoff), zero
// where x <= 0 when relu_mask (x is a ReLU output): dx [B, 2H, 2W, C] dense
__global__ void k_maxpool2_bwd(const bf16_t *x, int ldx, const bf16_t *dy, const bf16_t *dskip,
                               int ldskip, int skoff, int B, int H, int W, int C, int relu_mask,
                               bf16_t *dx) {
  const int C8 = C >> 3;
  const long n = (long)B * H * W * C8;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C8) * 8;
    const long pix = i / C8;
    const int w = (int)(pix % W), h = (int)((pix / W) % H), b = (int)(pix / ((long)W * H));
    float v[4][8], g[8];
    size_t pp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      pp[q] = (size_t)(b * 2 * H + 2 * h + (q >> 1)) * (2 * W) + 2 * w + (q & 1);
      unpack8(ld8(x + pp[q] * ldx + c), v[q]);
    }
    unpack8(ld8(dy + (size_t)pix * C + c), g);
    float m[8];
    bool taken[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      m[k] = fmaxf(fmaxf(v[0][k], v[1][k]), fmaxf(v[2][k], v[3][k]));
      taken[k] = false;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float sk[8], o[8];
      if (dskip) unpack8(ld8(dskip + pp[q] * ldskip + skoff + c), sk);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        o[k] = 0.f;
        if (!taken[k] && v[q][k] == m[k]) {
          o[k] = g[k];
          taken[k] = true;
        }
        if (dskip) o[k] += sk[k];
        if (relu_mask && !(v[q][k] > 0.f)) o[k] = 0.f;
      }
      st8(dx + pp[q] * C + c, pack8(o));
    }
  }
}

// nearest 2x upsampling: x [B, H, W, C] dense -> y [B, 2H, 2W, ldy] at channel offset yoff
__global__ void k_upsample2(const bf16_t *x, int B, int H, int W, int C, bf16_t *y, int ldy,
                            int yoff) {
  const int C8 = C >> 3;
  const long n = (long)B * 4 * H * W * C8;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C8) * 8;
    const long pix = i / C8;  // output pixel
    const int ww = (int)(pix % (2 * W)), hh = (int)((pix / (2 * W)) % (2 * H));
    const int b = (int)(pix / ((long)4 * W * H));
    st8(y + (size_t)pix * ldy + yoff + c, ld8(x + ((size_t)(b * H + hh / 2) * W + ww / 2) * C + c));
  }
}

// gradient of nearest 2x upsampling: dy [B, 2H, 2W, lddy] channels 0..C-1 ->
// dx [B, H, W, C], zero where mask <= 0 (mask [B, H, W, ldm], may be null)
__global__ void k_upsample2_bwd(const bf16_t *dy, int lddy, int B, int H, int W, int C,
                                const bf16_t *mask, int ldm, bf16_t *dx) {
  const int C8 = C >> 3;
  const long n = (long)B * H * W * C8;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C8) * 8;
    const long pix = i / C8;
    const int w = (int)(pix % W), h = (int)((pix / W) % H), b = (int)(pix / ((long)W * H));
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, t[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const size_t pp = (size_t)(b * 2 * H + 2 * h + (q >> 1)) * (2 * W) + 2 * w + (q & 1);
      unpack8(ld8(dy + pp * lddy + c), t);
#pragma unroll
      for (int k = 0; k < 8; ++k) s[k] += t[k];
    }
    if (mask) {
      float mk[8];
      unpack8(ld8(mask + (size_t)pix * ldm + c), mk);
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (!(mk[k] > 0.f)) s[k] = 0.f;
    }
    st8(dx + (size_t)pix * C + c, pack8(s));
  }
}

// ------------------------------------------------------------------- head
// z[p] = b + sum_c x[p, c] w[c]   (1x1 convolution to one logit, FP32)
__global__ void k_head_fwd(const bf16_t *x, int P, int C, const float *w, const float *b, float *z) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    float s = b[0];
    for (int c = 0; c < C; ++c) s += bf2f(x[(size_t)p * C + c]) * w[c];
    z[p] = s;
  }
}

// dx[p, c] = dz[p] w[c]; per-chunk partials of dw[c] = sum_p dz[p] x[p, c]
// and db = sum_p dz[p] into ws[chunk][C + 1]
__global__ void k_head_bwd(const bf16_t *x, int P, int C, const float *w, const float *dz,
                           bf16_t *dx, int chunk, float *ws) {
  const int z = blockIdx.x;
  const int pend = min(P, (z + 1) * chunk);
  __shared__ float red[33][33];
  const int c = threadIdx.x & 31, lane_p = threadIdx.x >> 5;  // 32 channels x 8 pixel lanes
  float s = 0.f, sb = 0.f;
  for (int p = z * chunk + lane_p; p < pend; p += 8) {
    const float g = dz[p];
    for (int cc = c; cc < C; cc += 32) {
      const float xv = bf2f(x[(size_t)p * C + cc]);
      // x is a ReLU output: its gradient is zero where x <= 0
      dx[(size_t)p * C + cc] = xv > 0.f ? f2bf(g * w[cc]) : (bf16_t)0;
      if (cc == c) s += g * xv;
    }
    sb += g;
  }
  red[lane_p][c] = s;
  if (c == 0) red[lane_p][32] = sb;
  __syncthreads();
  if (lane_p == 0) {
    float t = 0.f, tb = 0.f;
    for (int q = 0; q < 8; ++q) {
      t += red[q][c];
      tb += red[q][32];
    }
    if (c < C) ws[(size_t)z * (C + 1) + c] = t;
    if (c == 0) ws[(size_t)z * (C + 1) + C] = tb;
  }
}

// ------------------------------------------------------------------- loss
// class-weighted binary cross-entropy with logits, mean over n elements:
// dz = (pw t (sigma - 1) + (1 - t) sigma) / n; per-block loss partials
__global__ void k_bce(const float *z, const uint8_t *t, long n, float pw, float *dz, float *ws) {
  __shared__ float red[256];
  float s = 0.f;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float zi = z[i];
    const float tt = t[i] ? 1.f : 0.f;
    // log(1 + e^-z) and log(1 + e^z) without overflow
    const float sp_neg = fmaxf(-zi, 0.f) + log1pf(expf(-fabsf(zi)));
    const float sp_pos = sp_neg + zi;
    s += pw * tt * sp_neg + (1.f - tt) * sp_pos;
    const float sig = 1.f / (1.f + expf(-zi));
    dz[i] = (pw * tt * (sig - 1.f) + (1.f - tt) * sig) / (float)n;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) ws[blockIdx.x] = red[0];
}

// soft Dice over B samples of n_per logits each: per-(sample, chunk) partial
// sums of p t, p and t (p = sigma(z)), block (c, b) covering elements
// [c * chunk, (c + 1) * chunk) of sample b
constexpr int kDiceChunk = 4096;

__device__ __forceinline__ float block_sum256(float v, float *red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const float s = red[0];
  __syncthreads();
  return s;
}

__global__ void __launch_bounds__(256) k_dice_partial(const float *z, const uint8_t *t, long n_per,
                                                      float *ws) {
  __shared__ float red[256];
  const int c = blockIdx.x, b = blockIdx.y, nchunk = gridDim.x;
  const long lo = (long)c * kDiceChunk, hi = min(n_per, lo + kDiceChunk);
  const float *zb = z + (size_t)b * n_per;
  const uint8_t *tb = t + (size_t)b * n_per;
  float spt = 0.f, sp = 0.f, st = 0.f;
  for (long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const float p = 1.f / (1.f + expf(-zb[i]));
    const float tt = tb[i] ? 1.f : 0.f;
    spt += p * tt;
    sp += p;
    st += tt;
  }
  spt = block_sum256(spt, red);
  sp = block_sum256(sp, red);
  st = block_sum256(st, red);
  if (threadIdx.x == 0) {
    float *o = ws + ((size_t)b * nchunk + c) * 3;
    o[0] = spt;
    o[1] = sp;
    o[2] = st;
  }
}

// dz += -(w / B) (2 t (S + eps) - (2 I + eps)) / (S + eps)^2 p (1 - p), the
// sample's sums I = sum p t, S = sum p + sum t added in chunk order
__global__ void __launch_bounds__(256) k_dice_grad(const float *z, const uint8_t *t, long n_per,
                                                   int B, float w, float eps, const float *ws,
                                                   float *dz) {
  const int c = blockIdx.x, b = blockIdx.y, nchunk = gridDim.x;
  float I = 0.f, S = 0.f;
  for (int q = 0; q < nchunk; ++q) {
    const float *o = ws + ((size_t)b * nchunk + q) * 3;
    I += o[0];
    S += o[1] + o[2];
  }
  const float Se = S + eps, num = 2.f * I + eps, scale = -w / ((float)B * Se * Se);
  const long lo = (long)c * kDiceChunk, hi = min(n_per, lo + kDiceChunk);
  const float *zb = z + (size_t)b * n_per;
  const uint8_t *tb = t + (size_t)b * n_per;
  float *db = dz + (size_t)b * n_per;
  for (long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const float p = 1.f / (1.f + expf(-zb[i]));
    const float tt = tb[i] ? 1.f : 0.f;
    db[i] += scale * (2.f * tt * Se - num) * p * (1.f - p);
  }
}

// loss = w (1 - mean_b D_b), D_b = (2 I_b + eps) / (S_b + eps), in sample order
__global__ void k_dice_loss(const float *ws, int nchunk, int B, float w, float eps, float *loss) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float dsum = 0.f;
    for (int b = 0; b < B; ++b) {
      float I = 0.f, S = 0.f;
      for (int q = 0; q < nchunk; ++q) {
        const float *o = ws + ((size_t)b * nchunk + q) * 3;
        I += o[0];
        S += o[1] + o[2];
      }
      dsum += (2.f * I + eps) / (S + eps);
    }
    loss[0] = w * (1.f - dsum / (float)B);
  }
}

__global__ void k_sum_scaled(const float *ws, int m, float scale, float *out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < m; ++i) s += ws[i];
    out[0] = s * scale;
  }
}

// ------------------------------------------------------------------- adam
// w -= lr * mhat / (sqrt(vhat) + eps); BF16 copy of w, and for 3x3 weights
// [Cout][3][3][Cin] the transposed, flipped copy wt[Cin][3][3][Cout] with
// wt[c][ky][kx][o] = w[o][2-ky][2-kx][c] used by the data gradient
__global__ void k_adam(float *w, const float *g, float *m, float *v, long n, float lr, float b1,
                       float b2, float eps, float c1, float c2, bf16_t *wb, bf16_t *wt, int Cout,
                       int Cin) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    const bf16_t h = f2bf(wi);
    if (wb) wb[i] = h;
    if (wt) {
      const int c = (int)(i % Cin);
      const long r = i / Cin;
      const int kx = (int)(r % 3), ky = (int)((r / 3) % 3), o = (int)(r / 9);
      wt[(((size_t)c * 3 + (2 - ky)) * 3 + (2 - kx)) * Cout + o] = h;
    }
  }
}

__global__ void k_to_bf16(const float *x, long n, bf16_t *y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = f2bf(x[i]);
}

// dw[c] = sum_z ws[z][c], db = sum_z ws[z][C], in chunk order
__global__ void k_reduce_head(const float *ws, int nz, int C, float *dw, float *db) {
  for (int c = threadIdx.x; c <= C; c += blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < nz; ++z) s += ws[(size_t)z * (C + 1) + c];
    if (c < C) dw[c] = s;
    else db[0] = s;
  }
}

int grid_1d(long n, int block) {
  long b = (n + block - 1) / block;
  return (int)(b < 1 ? 1 : (b > 4 * 1216 ? 4 * 1216 : b));
}

}  // namespace

// ======================================================================= ABI
extern "C" {

int cem_sg_conv3x3(const void *x, int B, int H, int W, int Cin, int ldx, const void *w,
                   const float *bias, int Cout, int relu, const void *mask, int ldmask, void *y,
                   int ldy, int yoff, void *stream) {
  if (!x || !w || !y || B < 1 || H < 1 || W < 1 || Cin < 8 || (Cin & 7) || ldx < Cin ||
      (ldx & 7) || Cout < 2 || (Cout & 1) || ldy < yoff + Cout || (yoff & 1) ||
      (mask && (ldmask < Cout || (ldmask & 1))))
    return CEM_SG_ERR_ARG;
  ConvArgs a;
  a.x = (const bf16_t *)x;
  a.w = (const bf16_t *)w;
  a.bias = bias;
  a.y = (bf16_t *)y;
  a.B = B; a.H = H; a.W = W; a.Cin = Cin; a.ldx = ldx; a.N = Cout; a.K = 9 * Cin;
  a.relu = relu; a.ldy = ldy; a.yoff = yoff; a.P = B * H * W;
  a.mask = (const bf16_t *)mask;
  a.ldm = ldmask;
  cudaStream_t st = (cudaStream_t)stream;
  if (g_use_tc) {
    cudaError_t e = Cout > 128 ? launch_conv_tc<256>(a, st)
                  : Cout > 64 ? launch_conv_tc<128>(a, st)
                  : Cout > 32 ? launch_conv_tc<64>(a, st) : launch_conv_tc<32>(a, st);
    return e == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
  }
  dim3 grid((a.P + FBM - 1) / FBM, (Cout + FBN - 1) / FBN);
  k_conv3x3<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
}

long cem_sg_wgrad_workspace(int B, int H, int W, int Cin, int Cout) {
  const long P = (long)B * H * W;
  long splits = (P + 4095) / 4096;
  if (splits > 512) splits = 512;
  return splits * (long)Cout * 9 * Cin * 4 + (long)Cout * 4 * 1024;
}

int cem_sg_conv3x3_wgrad(const void *x, int ldx, const void *dy, int lddy, int B, int H, int W,
                         int Cin, int Cout, float *dw, float *db, void *ws, long ws_bytes,
                         void *stream) {
  if (!x || !dy || !dw || !ws || B < 1 || H < 1 || W < 1 || Cin < 8 || (Cin & 7) ||
      (ldx & 7) || ldx < Cin || Cout < 8 || (Cout & 7) || lddy < Cout || (lddy & 7))
    return CEM_SG_ERR_ARG;
  if (ws_bytes < cem_sg_wgrad_workspace(B, H, W, Cin, Cout)) return CEM_SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  WgradArgs a;
  a.x = (const bf16_t *)x;
  a.dy = (const bf16_t *)dy;
  a.ws = (float *)ws;
  a.B = B; a.H = H; a.W = W; a.Cin = Cin; a.ldx = ldx; a.lddy = lddy; a.N = Cout;
  a.K = 9 * Cin; a.P = B * H * W;
  int splits = (a.P + 4095) / 4096;
  if (splits > 512) splits = 512;
  a.chunk = ((a.P + splits - 1) / splits + GBK - 1) / GBK * GBK;
  splits = (a.P + a.chunk - 1) / a.chunk;
  const long nw = (long)Cout * a.K;
  if (g_use_tc) {
    // tcgen05: dW^T tiles of 128 k' x BN outputs; bias sums by a separate
    // coalesced reduction into the workspace after the weight partials
    a.wsb = nullptr;
    cudaError_t e = Cout > 128 ? launch_wgrad_tc<256>(a, splits, st)
                  : Cout > 64 ? launch_wgrad_tc<128>(a, splits, st)
                              : launch_wgrad_tc<64>(a, splits, st);
    if (e != cudaSuccess) return CEM_SG_ERR_CUDA;
    k_reduce_splits<<<grid_1d(nw, 256), 256, 0, st>>>(a.ws, splits, nw, dw);
    if (db) {
      // more pixel chunks than the weight partials use: the sums are a pure
      // bandwidth pass (at most 608 chunks, four per SM; the workspace holds 1024)
      float *wsb = a.ws + (size_t)splits * Cout * a.K;
      const long bs = (a.P + 2047) / 2048;
      const int bsplits = (int)(bs < 1 ? 1 : (bs > 608 ? 608 : bs));
      const int bch = (a.P + bsplits - 1) / bsplits;
      k_colsum8<<<bsplits, 256, 0, st>>>(a.dy, a.P, Cout, lddy, bch, wsb);
      k_reduce_splits<<<grid_1d(Cout, 128), 128, 0, st>>>(wsb, bsplits, Cout, db);
    }
    return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
  }
  a.wsb = db ? a.ws + (size_t)splits * Cout * a.K : nullptr;
  dim3 grid((Cout + GBM - 1) / GBM, (a.K + GBN - 1) / GBN, splits);
  k_conv3x3_wgrad<<<grid, 256, 0, st>>>(a);
  k_reduce_splits<<<grid_1d(nw, 256), 256, 0, st>>>(a.ws, splits, nw, dw);
  if (db) k_reduce_splits<<<grid_1d(Cout, 128), 128, 0, st>>>(a.wsb, splits, Cout, db);
  return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
}

int cem_sg_relu_bwd(void *dy, int lddy, const void *y, int ldy, long P, int C, void *stream) {
  if (!dy || !y || P < 0 || C < 1 || lddy < C || ldy < C) return CEM_SG_ERR_ARG;
  k_relu_bwd<<<grid_1d(P * C, 256), 256, 0, (cudaStream_t)stream>>>((bf16_t *)dy, lddy,
                                                                    (const bf16_t *)y, ldy, P, C);
  return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
}

int cem_sg_maxpool2(const void *x, int ldx, int B, int H, int W, int C, void *y, void *stream) {
  if (!x || !y || B < 1 || H < 1 || W < 1 || C < 8 || (C & 7) || ldx < C || (ldx & 7))
    return CEM_SG_ERR_ARG;
  const long n = (long)B * H * W * (C >> 3);
  k_maxpool2<<<grid_1d(n, 256), 256, 0, (cudaStream_t)stream>>>((const bf16_t *)x, ldx, B, H, W, C,
                                                               (bf16_t *)y);
  return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
}

int cem_sg_maxpool2_bwd(const void *x, int ldx, const void *dy, const void *dskip, int ldskip,
                        int skoff, int B, int H, int W, int C, int relu_mask, void *dx,
                        void *stream) {
  if (!x || !dy || !dx || B < 1 || H < 1 || W < 1 || C < 8 || (C & 7) || ldx < C || (ldx & 7) ||
      (dskip && (ldskip < skoff + C || (ldskip & 7) || (skoff & 7))))
    return CEM_SG_ERR_ARG;
  const long n = (long)B * H * W * (C >> 3);
  k_maxpool2_bwd<<<grid_1d(n, 256), 256, 0, (cudaStream_t)stream>>>(
      (const bf16_t *)x, ldx, (const bf16_t *)dy, (const bf16_t *)dskip, ldskip, skoff, B, H, W, C,
      relu_mask, (bf16_t *)dx);
  return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
}

int cem_sg_upsample2(const void *x, int B, int H, int W, int C, void *y, int ldy, int yoff,
                     void *stream) {
  if (!x || !y || B < 1 || H < 1 || W < 1 || C < 8 || (C & 7) || ldy < yoff + C || (ldy & 7) ||
      (yoff & 7))
    return CEM_SG_ERR_ARG;
  const long n = (long)B * 4 * H * W * (C >> 3);
  k_upsample2<<<grid_1d(n, 256), 256, 0, (cudaStream_t)stream>>>((const bf16_t *)x, B, H, W, C,
                                                                (bf16_t *)y, ldy, yoff);
  return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
}

int cem_sg_upsample2_bwd(const void *dy, int lddy, int B, int H, int W, int C, const void *mask,
                         int ldmask, void *dx, void *stream) {
  if (!dy || !dx || B < 1 || H < 1 || W < 1 || C < 8 || (C & 7) || lddy < C || (lddy & 7) ||
      (mask && (ldmask < C || (ldmask & 7))))
    return CEM_SG_ERR_ARG;
  const long n = (long)B * H * W * (C >> 3);
  k_upsample2_bwd<<<grid_1d(n, 256), 256, 0, (cudaStream_t)stream>>>(
      (const bf16_t *)dy, lddy, B, H, W, C, (const bf16_t *)mask, ldmask, (bf16_t *)dx);
  return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
}

int cem_sg_head_fwd(const void *x, int P, int C, const float *w, const float *b, float *z,
                    void *stream) {
  if (!x || !w || !b || !z || P < 1 || C < 1) return CEM_SG_ERR_ARG;
  k_head_fwd<<<grid_1d(P, 256), 256, 0, (cudaStream_t)stream>>>((const bf16_t *)x, P, C, w, b, z);
  return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
}

long cem_sg_head_workspace(int P, int C) {
  const long nz = (P + 4095) / 4096;
  return nz * (C + 1) * 4;
}

int cem_sg_head_bwd(const void *x, int P, int C, const float *w, const float *dz, void *dx,
                    float *dw, float *db, void *ws, long ws_bytes, void *stream) {
  if (!x || !w || !dz || !dx || !dw || !db || !ws || P < 1 || C < 1 || C > 32)
    return CEM_SG_ERR_ARG;
  if (ws_bytes < cem_sg_head_workspace(P, C)) return CEM_SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int chunk = 4096, nz = (P + chunk - 1) / chunk;
  float *wsf = (float *)ws;
  k_head_bwd<<<nz, 256, 0, st>>>((const bf16_t *)x, P, C, w, dz, (bf16_t *)dx, chunk, wsf);
  k_reduce_head<<<1, 64, 0, st>>>(wsf, nz, C, dw, db);
  return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
}

long cem_sg_bce_workspace(long n) { return 4 * 1216 * 4 + 16; }

int cem_sg_bce(const float *z, const unsigned char *t, long n, float pos_weight, float *dz,
               float *loss, void *ws, long ws_bytes, void *stream) {
  if (!z || !t || !dz || !loss || !ws || n < 1) return CEM_SG_ERR_ARG;
  if (ws_bytes < cem_sg_bce_workspace(n)) return CEM_SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int g = grid_1d(n, 256);
  k_bce<<<g, 256, 0, st>>>(z, t, n, pos_weight, dz, (float *)ws);
  k_sum_scaled<<<1, 32, 0, st>>>((const float *)ws, g, 1.f / (float)n, loss);
  return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
}

long cem_sg_dice_workspace(int B, long n_per) {
  if (B < 1 || n_per < 1) return 0;
  return (long)B * ((n_per + kDiceChunk - 1) / kDiceChunk) * 3 * 4;
}

int cem_sg_dice(const float *z, const unsigned char *t, int B, long n_per, float weight, float eps,
                float *dz, float *loss, void *ws, long ws_bytes, void *stream) {
  if (!z || !t || !dz || !loss || !ws || B < 1 || n_per < 1 || !(eps > 0.f)) return CEM_SG_ERR_ARG;
  if (ws_bytes < cem_sg_dice_workspace(B, n_per)) return CEM_SG_ERR_ARG;
  const long nchunk = (n_per + kDiceChunk - 1) / kDiceChunk;
  if (nchunk > 65535 || B > 65535) return CEM_SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const dim3 grid((unsigned)nchunk, (unsigned)B);
  k_dice_partial<<<grid, 256, 0, st>>>(z, t, n_per, (float *)ws);
  k_dice_grad<<<grid, 256, 0, st>>>(z, t, n_per, B, weight, eps, (const float *)ws, dz);
  k_dice_loss<<<1, 32, 0, st>>>((const float *)ws, (int)nchunk, B, weight, eps, loss);
  return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
}

int cem_sg_adam(float *w, const float *g, float *m, float *v, long n, float lr, float beta1,
                float beta2, float eps, int step, void *w_bf16, void *wt_bf16, int Cout, int Cin,
                void *stream) {
  if (!w || !g || !m || !v || n < 1 || step < 1 || !(lr >= 0.f)) return CEM_SG_ERR_ARG;
  if (wt_bf16 && (Cout < 1 || Cin < 1 || (long)Cout * 9 * Cin != n)) return CEM_SG_ERR_ARG;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<grid_1d(n, 256), 256, 0, (cudaStream_t)stream>>>(
      w, g, m, v, n, lr, beta1, beta2, eps, c1, c2, (bf16_t *)w_bf16, (bf16_t *)wt_bf16, Cout, Cin);
  return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
}

int cem_sg_set_gemm_path(int use_tcgen05) {
  g_use_tc = use_tcgen05 ? 1 : 0;
  return CEM_SG_OK;
}

int cem_sg_timeouts(int *count) {
  if (!count) return CEM_SG_ERR_ARG;
  return cudaMemcpyFromSymbol(count, g_tc_timeouts, sizeof(int)) == cudaSuccess ? CEM_SG_OK
                                                                             : CEM_SG_ERR_CUDA;
}

int cem_sg_to_bf16(const float *x, long n, void *y, void *stream) {
  if (!x || !y || n < 0) return CEM_SG_ERR_ARG;
  k_to_bf16<<<grid_1d(n, 256), 256, 0, (cudaStream_t)stream>>>(x, n, (bf16_t *)y);
  return cudaGetLastError() == cudaSuccess ? CEM_SG_OK : CEM_SG_ERR_CUDA;
}

}  // extern "C"
