// Toeplitz products of one multigrid level on the 5th-generation tensor cores
// (tcgen05 + TMEM + TMA), sm_103a.
//
// For a level grid X (n2 rows y, n1 columns x) the operator of Eq. (AxAy)
// needs four dense products, each a GEMM with one Toeplitz factor:
//     acc0 = X  A_x^T   (rows of X times A_x)        acc1 = X  A_x
//     acc2 = A_y X                                  acc3 = A_y^T X
// One CTA owns a 128 x 128 output tile and keeps all four FP32 accumulators
// in tensor memory (4 x 128 columns = the whole 512-column TMEM).  A 64-deep
// K-block of a Toeplitz factor depends only on the block-diagonal offset
// delta = (output block start) - (K block start), so the factor is stored as
// a bank of 128 x 64 tiles, one per offset (O(n) tiles, never an n x n
// matrix), built once per level from the generator t_d and streamed by TMA
// like any other operand.  Blocks whose Toeplitz tile is identically zero
// (above the super-diagonal) are skipped: each accumulator visits only the
// K-blocks its triangle touches.  The epilogue scales by the coefficient
// fields and adds the mass term: kx = cm M + dp acc0 + dm acc1 + ep acc2 + em acc3.
//
// Warp roles (192 threads): warp 0 issues TMA loads, warp 1 (one elected
// lane) issues tcgen05.mma, warps 2-5 drain TMEM in the epilogue.  Every
// mbarrier wait is bounded; on timeout the CTA raises a device error flag,
// drains its in-flight copies and MMAs, frees TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <cstring>

#include "tc_gemm.h"

namespace fde {
namespace tc {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int STAGES = 6;
constexpr int TILE_BYTES = BM * BK * 2;  // 16 KB: 128 rows x 128 B
constexpr int NUM_THREADS = 192;
constexpr uint32_t TMEM_COLS = 512;
constexpr size_t SMEM_BYTES = (size_t)STAGES * 2 * TILE_BYTES + 1024 /*align*/ + 256 /*bars*/;

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait (about one second): false on timeout or when another role of
// the CTA already gave up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  uint64_t t0 = 0;
  for (uint32_t i = 0;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255) == 255) {
      if (*abort) return false;
      const uint64_t t = global_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > 1000000000ull) break;
      __nanosleep(64);
    }
  }
  *abort = 1;
  return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of sm_100-class tensor cores
  d |= (uint64_t)2 << 61;  // 128-byte swizzle
  return d;
}
// kind::f16 instruction descriptor: D F32, A/B BF16 or F16, A K-major,
// B K-major or MN-major, N = 128, M = 128
__host__ __device__ constexpr uint32_t make_idesc(bool b_mn_major, bool f16) {
  return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) |
         ((b_mn_major ? 1u : 0u) << 16) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// ---------------------------------------------------------------- job list
// The K loop of a tile visits, in order: x-direction blocks (acc 0 / acc 1)
// then y-direction blocks (acc 2 / acc 3), skipping identically-zero blocks.
// Block offset delta = out0 - k0: acc 0/2 (lower Hessenberg) is nonzero for
// delta >= -128, acc 1/3 (its transpose) for delta <= 64.
struct JobIter {
  int i0, j0, nkx, nky;
  int phase = 0, kb = 0, sub = 0;  // phase 0: x, 1: y, 2: done
  __device__ bool next(int& acc, int& k0, int& delta) {
    while (phase < 2) {
      const int nk = phase == 0 ? nkx : nky;
      const int out0 = phase == 0 ? i0 : j0;
      if (kb >= nk) {
        ++phase;
        kb = 0;
        sub = 0;
        continue;
      }
      k0 = kb * BK;
      delta = out0 - k0;
      const int s = sub;
      if (++sub == 2) {
        sub = 0;
        ++kb;
      }
      if (s == 0 && delta >= -128) { acc = phase * 2; return true; }
      if (s == 1 && delta <= 64) { acc = phase * 2 + 1; return true; }
    }
    return false;
  }
};

struct KParams {
  const float* M;  // mass term source (may be null)
  float cm;
  const float *dp, *dm, *ep, *em;
  float* kx;
  int n1, n2;
  int rowL_x, rowU_x, rowL_y, rowU_y;  // first bank row of each bank
  float inv_scale;                     // 1 / bank scale
  int* err;
};

__global__ void __launch_bounds__(NUM_THREADS, 1)
toeplitz_gemm_kernel(const __grid_constant__ CUtensorMap mapXa,
                     const __grid_constant__ CUtensorMap mapXb,
                     const __grid_constant__ CUtensorMap mapBank, const KParams kp,
                     uint32_t idesc_x, uint32_t idesc_y) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* tilesA = base;                         // STAGES x 16 KB
  unsigned char* tilesB = base + STAGES * TILE_BYTES;   // STAGES x 16 KB
  uint64_t* bars = (uint64_t*)(base + 2 * STAGES * TILE_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* accbar = bars + 2 * STAGES;
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * BN, j0 = blockIdx.y * BM;
  const int nkx = (kp.n1 + BK - 1) / BK, nky = (kp.n2 + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(accbar), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      JobIter it{i0, j0, nkx, nky};
      int acc, k0, delta, n = 0;
      int last_parity[STAGES];
      bool issued[STAGES];
      for (int s = 0; s < STAGES; ++s) issued[s] = false;
      while (!*abort_flag && it.next(acc, k0, delta)) {
        const int s = n % STAGES;
        const uint32_t ph = (uint32_t)(n / STAGES) & 1u;
        if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u, abort_flag)) break;
        const uint32_t fb = smem_u32(&full[s]);
        mbar_expect_tx(fb, 2 * TILE_BYTES);
        const uint32_t dA = smem_u32(tilesA + s * TILE_BYTES);
        const uint32_t dB = smem_u32(tilesB + s * TILE_BYTES);
        if (acc < 2) {
          const int row = acc == 0 ? kp.rowL_x + ((delta + 128) / 64) * BM
                                   : kp.rowU_x + ((64 - delta) / 64) * BM;
          tma_load_2d(dA, &mapXa, k0, j0, fb);      // X[j0.., k0..]   (K-major)
          tma_load_2d(dB, &mapBank, 0, row, fb);    // Toeplitz tile   (K-major)
        } else {
          const int row = acc == 2 ? kp.rowL_y + ((delta + 128) / 64) * BM
                                   : kp.rowU_y + ((64 - delta) / 64) * BM;
          tma_load_2d(dA, &mapBank, 0, row, fb);            // Toeplitz tile (K-major)
          tma_load_2d(dB, &mapXb, i0, k0, fb);              // X[k0.., i0..i0+63]  (MN-major)
          tma_load_2d(dB + TILE_BYTES / 2, &mapXb, i0 + 64, k0, fb);
        }
        issued[s] = true;
        last_parity[s] = (int)ph;
        ++n;
      }
      // drain: every issued copy has landed before the CTA can exit
      const uint64_t t0 = global_ns();
      for (int s = 0; s < STAGES; ++s)
        if (issued[s]) {
          while (!mbar_try(smem_u32(&full[s]), (uint32_t)last_parity[s]))
            if (global_ns() - t0 > 1000000000ull) break;
        }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      JobIter it{i0, j0, nkx, nky};
      int acc, k0, delta, n = 0;
      bool started[4] = {false, false, false, false};
      while (!*abort_flag && it.next(acc, k0, delta)) {
        const int s = n % STAGES;
        const uint32_t ph = (uint32_t)(n / STAGES) & 1u;
        if (!mbar_wait(smem_u32(&full[s]), ph, abort_flag)) break;
        fence_after();
        const uint32_t aA = smem_u32(tilesA + s * TILE_BYTES);
        const uint32_t aB = smem_u32(tilesB + s * TILE_BYTES);
        const uint32_t d = tmem + (uint32_t)(acc * BN);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t da = smem_desc(aA + kk * 32, 16, 1024);
          uint64_t db;
          uint32_t idesc;
          if (acc < 2) {
            db = smem_desc(aB + kk * 32, 16, 1024);
            idesc = idesc_x;
          } else {
            db = smem_desc(aB + kk * 2048, TILE_BYTES / 2, 1024);
            idesc = idesc_y;
          }
          mma_f16(d, da, db, idesc, (started[acc] || kk > 0) ? 1u : 0u);
        }
        started[acc] = true;
        mma_commit(smem_u32(&empty[s]));
        ++n;
      }
      mma_commit(smem_u32(accbar));  // completes when every MMA above has completed
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // Warp w may read TMEM lanes 32 (w % 4) .. +31, i.e. output rows
    // 32 g .. 32 g + 31.  Per 32-column chunk the four accumulators go through
    // a padded per-warp staging area (the operand buffers are idle once the
    // accumulator barrier has fired) so that afterwards lane = column and every
    // global load/store of the epilogue is one 128-byte row segment.
    const int g = warp & 3;
    // one lane per warp waits for the accumulators (backing off between polls so
    // the waiting warps do not compete with TMA completions on the barrier unit)
    int okw = 1;
    if (lane == 0) {
      const uint64_t t0 = global_ns();
      while (!mbar_try(smem_u32(accbar), 0)) {
        if (*abort_flag) { okw = 0; break; }
        if (global_ns() - t0 > 1000000000ull) { *abort_flag = 1; okw = 0; break; }
        __nanosleep(256);
      }
    }
    const bool ok = __shfl_sync(0xffffffffu, okw, 0) != 0;
    fence_after();
    if (ok && !*abort_flag) {
      float* stg = reinterpret_cast<float*>(tilesA) + (warp - 2) * (4 * 32 * 33);
      const uint32_t tl = tmem + ((uint32_t)(g * 32) << 16);
      for (int cb = 0; cb < BN; cb += 32) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          float v[32];
          tmem_ld32(tl + a * BN + cb, v);
          tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < 32; ++q) stg[(a * 32 + lane) * 33 + q] = v[q];
        }
        __syncwarp();
        const int col = i0 + cb + lane;
        if (col < kp.n1) {
          for (int rr = 0; rr < 32; ++rr) {
            const int row = j0 + g * 32 + rr;
            if (row >= kp.n2) break;
            const size_t idx = (size_t)row * kp.n1 + col;
            float v = kp.inv_scale * (kp.dp[idx] * stg[(0 * 32 + rr) * 33 + lane] +
                                      kp.dm[idx] * stg[(1 * 32 + rr) * 33 + lane] +
                                      kp.ep[idx] * stg[(2 * 32 + rr) * 33 + lane] +
                                      kp.em[idx] * stg[(3 * 32 + rr) * 33 + lane]);
            if (kp.M) v += kp.cm * kp.M[idx];
            kp.kx[idx] = v;
          }
        }
        __syncwarp();
      }
    }
  }
  fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicExch(kp.err, 1);
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

// ---------------------------------------------------------------- helpers
template <typename H>
__device__ __forceinline__ H to_h(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_h<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_h<__half>(float v) { return __float2half_rn(v); }

// bank tile (b, i, k): L bank t[delta + i - k], U bank t[-delta + k - i],
// delta = -128 + 64 b (L) or 64 - 64 b (U); zero outside d in [-1, n-1]
template <typename H>
__global__ void bank_kernel(const double* __restrict__ t, int n, int ntL, int ntU, float scale,
                            H* bankL, H* bankU) {
  const size_t totL = (size_t)ntL * BM * BK, tot = totL + (size_t)ntU * BM * BK;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot;
       e += (size_t)gridDim.x * blockDim.x) {
    const bool upper = e >= totL;
    const size_t f = upper ? e - totL : e;
    const int b = (int)(f / (BM * BK)), i = (int)((f / BK) % BM), k = (int)(f % BK);
    int d;
    if (!upper) d = (-128 + 64 * b) + i - k;
    else d = -(64 - 64 * b) + k - i;
    const float v = (d >= -1 && d <= n - 1) ? (float)(scale * t[d + 1]) : 0.f;
    (upper ? bankU : bankL)[f] = to_h<H>(v);
  }
}

template <typename H>
__global__ void pack_kernel(const float* __restrict__ X, int n1, int n2, int ld, H* out) {
  const size_t N = (size_t)n1 * n2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n1), j = (int)(e / n1);
    out[(size_t)j * ld + i] = to_h<H>(X[e]);
  }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled get_encoder() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
  }
  return fn;
}

struct Maps {
  CUtensorMap xa, xb, bank;
  int rowL_x, rowU_x, rowL_y, rowU_y;
  int* err;
};

static int encode(CUtensorMap* m, CUtensorMapDataType dt, void* ptr, uint64_t d0, uint64_t d1,
                  uint64_t stride_bytes, uint32_t b0, uint32_t b1) {
  EncodeTiled enc = get_encoder();
  if (!enc) return 10;
  cuuint64_t dims[2] = {d0, d1};
  cuuint64_t strides[1] = {stride_bytes};
  cuuint32_t box[2] = {b0, b1};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, dt, 2, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : 11;
}

int level_create(ToeplitzGemmLevel* L, int n1, int n2, int prec, bool mass) {
  L->n1 = n1;
  L->n2 = n2;
  L->prec = prec;
  L->ld = (n1 + 63) / 64 * 64;
  const size_t xbytes = (size_t)n2 * L->ld * 2;
  if (cudaMalloc(&L->xa, xbytes) != cudaSuccess) return 1;
  if (cudaMemset(L->xa, 0, xbytes) != cudaSuccess) return 1;
  if (mass) {
    if (cudaMalloc(&L->xb, xbytes) != cudaSuccess) return 1;
    if (cudaMemset(L->xb, 0, xbytes) != cudaSuccess) return 1;
  }
  // bank tile counts: L tiles for delta = -128 .. (last output block start),
  // U tiles for delta = 64 .. -(last K block start)
  auto ntl = [](int n) { return ((n + BN - 1) / BN - 1) * (BN / BK) + 3; };
  auto ntu = [](int n) { return (n + BK - 1) / BK + 1; };
  const int tLx = ntl(n1), tUx = ntu(n1), tLy = ntl(n2), tUy = ntu(n2);
  L->tiles_x = tLx + tUx;
  L->tiles_y = tLy + tUy;
  const size_t bank_rows = (size_t)(L->tiles_x + L->tiles_y) * BM;
  if (cudaMalloc(&L->bank, bank_rows * BK * 2) != cudaSuccess) return 1;
  Maps hm;
  const CUtensorMapDataType dt =
      prec == kFP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  int r = encode(&hm.xa, dt, L->xa, n1, n2, (uint64_t)L->ld * 2, BK, BM);
  if (r) return r;
  r = encode(&hm.xb, dt, mass ? L->xb : L->xa, n1, n2, (uint64_t)L->ld * 2, BK, BK);
  if (r) return r;
  r = encode(&hm.bank, dt, L->bank, BK, bank_rows, BK * 2, BK, BM);
  if (r) return r;
  hm.rowL_x = 0;
  hm.rowU_x = tLx * BM;
  hm.rowL_y = (tLx + tUx) * BM;
  hm.rowU_y = (tLx + tUx + tLy) * BM;
  if (cudaMalloc(&hm.err, sizeof(int)) != cudaSuccess) return 1;
  if (cudaMemset(hm.err, 0, sizeof(int)) != cudaSuccess) return 1;
  Maps* hp = new Maps(hm);
  L->maps = hp;
  if (cudaFuncSetAttribute(toeplitz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)SMEM_BYTES) != cudaSuccess)
    return 12;
  L->built = true;
  return 0;
}

int level_setup(ToeplitzGemmLevel* L, const double* tx, const double* ty, cudaStream_t st) {
  if (!L->built) return 20;
  Maps* m = (Maps*)L->maps;
  const float scale = L->prec == kFP16 ? 1024.f : 1.f;
  const int tLx = m->rowU_x / BM, tUx = (m->rowL_y - m->rowU_x) / BM;
  const int tLy = (m->rowU_y - m->rowL_y) / BM, tUy = L->tiles_y - tLy;
  const size_t tile = (size_t)BM * BK;
  if (L->prec == kFP16) {
    __half* b = (__half*)L->bank;
    bank_kernel<__half><<<512, 256, 0, st>>>(tx, L->n1, tLx, tUx, scale, b, b + tLx * tile);
    bank_kernel<__half><<<512, 256, 0, st>>>(ty, L->n2, tLy, tUy, scale,
                                             b + (size_t)(tLx + tUx) * tile,
                                             b + (size_t)(tLx + tUx + tLy) * tile);
  } else {
    __nv_bfloat16* b = (__nv_bfloat16*)L->bank;
    bank_kernel<__nv_bfloat16><<<512, 256, 0, st>>>(tx, L->n1, tLx, tUx, scale, b, b + tLx * tile);
    bank_kernel<__nv_bfloat16><<<512, 256, 0, st>>>(ty, L->n2, tLy, tUy, scale,
                                                    b + (size_t)(tLx + tUx) * tile,
                                                    b + (size_t)(tLx + tUx + tLy) * tile);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : 21;
}

int level_products(ToeplitzGemmLevel* L, const float* xin_x, const float* xin_y, const float* M,
                   double cm, const float* dp, const float* dm, const float* ep, const float* em,
                   float* kx, cudaStream_t st) {
  if (!L->built) return 30;
  Maps* m = (Maps*)L->maps;
  const int n1 = L->n1, n2 = L->n2;
  const size_t N = (size_t)n1 * n2;
  int g = (int)((N + 255) / 256);
  if (g > 152 * 16) g = 152 * 16;
  const bool two = L->xb != nullptr;
  if (L->prec == kFP16) {
    pack_kernel<__half><<<g, 256, 0, st>>>(xin_x, n1, n2, L->ld, (__half*)L->xa);
    if (two) pack_kernel<__half><<<g, 256, 0, st>>>(xin_y, n1, n2, L->ld, (__half*)L->xb);
  } else {
    pack_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(xin_x, n1, n2, L->ld, (__nv_bfloat16*)L->xa);
    if (two)
      pack_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(xin_y, n1, n2, L->ld,
                                                    (__nv_bfloat16*)L->xb);
  }
  KParams kp;
  kp.M = M;
  kp.cm = (float)cm;
  kp.dp = dp;
  kp.dm = dm;
  kp.ep = ep;
  kp.em = em;
  kp.kx = kx;
  kp.n1 = n1;
  kp.n2 = n2;
  kp.rowL_x = m->rowL_x;
  kp.rowU_x = m->rowU_x;
  kp.rowL_y = m->rowL_y;
  kp.rowU_y = m->rowU_y;
  kp.inv_scale = L->prec == kFP16 ? 1.f / 1024.f : 1.f;
  kp.err = m->err;
  const bool f16 = L->prec == kFP16;
  dim3 grid((n1 + BN - 1) / BN, (n2 + BM - 1) / BM);
  toeplitz_gemm_kernel<<<grid, NUM_THREADS, SMEM_BYTES, st>>>(
      m->xa, m->xb, m->bank, kp, make_idesc(false, f16), make_idesc(true, f16));
  return cudaGetLastError() == cudaSuccess ? 0 : 31;
}

int level_error(ToeplitzGemmLevel* L) {
  if (!L->built) return 0;
  Maps* m = (Maps*)L->maps;
  int e = 0;
  cudaMemcpy(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost);
  return e;
}

void level_destroy(ToeplitzGemmLevel* L) {
  if (L->maps) {
    Maps* m = (Maps*)L->maps;
    cudaFree(m->err);
    delete m;
  }
  cudaFree(L->xa);
  cudaFree(L->xb);
  cudaFree(L->bank);
  L->xa = L->xb = L->bank = L->maps = nullptr;
  L->built = false;
}

}  // namespace tc
}  // namespace fde
