// Toeplitz products of one multigrid level on the 5th-generation tensor cores
// (tcgen05 + TMEM + TMA), sm_103a.
//
// For a level grid X (n2 rows y, n1 columns x) the operator of Eq. (AxAy)
// needs four dense products with one Toeplitz factor each:
//     X A_x^T and X A_x          (x direction; output rows j, columns i)
//     A_y X  and A_y^T X         (y direction)
// Two launches cover them.  An x-CTA owns a 128 (j) x 256 (i) output tile and
// accumulates X A_x^T and X A_x in two FP32 TMEM accumulators of 256 columns
// (the whole 512-column TMEM).  A y-CTA owns a 128 (i) x 256 (j) tile of the
// TRANSPOSED y products, D[i][j] = sum_k X[k][i] A_y[j][k] (and A_y[k][j]):
// its A operand is X read MN-major, and its TMEM lanes are grid columns, so
// its epilogue stores are coalesced without staging.
//
// Operands.  The X tiles (128 x 64, 16-bit) are streamed by TMA.  The Toeplitz
// tiles (256 x 64) are never stored: a 64-deep K block of A_gamma at output
// offset delta is B[r][k] = t[delta + r - k] (or t[-delta + k - r] for the
// transpose), so eight "synthesis" warps -- the epilogue warps, idle during the
// main loop -- stage a 320-element window of the O(n) generator t in shared
// memory and write the tile in the 128-byte-swizzled K-major layout the
// tensor core reads, while the previous block multiplies.  Blocks whose tile
// is identically zero (above the super-diagonal) are skipped.
//
// Precision.  kBF16 / kFP16: one product per block (16-bit operands, FP32
// accumulation).  kBF16X3: X = X_hi + X_lo and t = t_hi + t_lo split into
// BF16 pairs and three products (hi hi, lo hi, hi lo) accumulated in FP32:
// ~16-bit operands, which keeps the multigrid preconditioner as effective as
// an FP32 one (the residual b - K x of a smooth x cancels heavily).
//
// Roles (320 threads): warp 0 issues TMA, warp 1 (one lane) issues tcgen05.mma,
// warps 2-9 synthesise Toeplitz tiles and then drain TMEM in the epilogue (two
// warps per TMEM lane group, each taking half of the tile's columns).
// Every mbarrier wait is bounded (about one second); on timeout the CTA raises
// a device error flag, drains its copies and MMAs, frees TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <cstring>

#include "tc_gemm.h"

namespace fde {
namespace tc {

// Output tiles of 128 x 240: at n = 2047 a launch has 9 x 16 = 144 CTAs for
// the 152 SMs (256-wide tiles would leave 24 idle), and the smaller Toeplitz
// operand leaves room for a third X-tile stage.
constexpr int BM = 128, BN = 240, BK = 64;
constexpr int ACC_COLS = 256;          // TMEM columns between the two accumulators
constexpr int BH = 128;                // epilogue column split: [0, BH) and [BH, BN)
constexpr int A_BYTES = BM * BK * 2;   // 16 KB
constexpr int B_BYTES = BN * BK * 2;   // 30 KB
constexpr int NUM_THREADS = 320;  // 2 + 8 warps
constexpr int NSYN = 8;            // synthesis / epilogue warps
constexpr uint32_t TMEM_COLS = 512;
constexpr int GEN_OFF = 320;           // zero padding in front of the generator copy
constexpr int GEN_PAD = 1024;          // total padding elements
// A job's Toeplitz tile reads generator entries base0 - 255 .. base0 + 68 of
// one copy (forward or reversed); the producer streams the 16-byte aligned
// window [ws, ws + WIN), ws = (base0 - 256) rounded down to 8 entries, into
// the stage's window buffer with one bulk copy per term.
constexpr int WIN = 336;               // entries (16-bit) per window
constexpr int WIN_BYTES = WIN * 2;     // 672: a multiple of 16

// Two rings: the X tiles (A operand) and the generator windows in SA slots,
// filled by TMA up to SA jobs ahead; the synthesised Toeplitz tiles (B
// operand) in SB slots.  An X slot is released when the job's MMAs complete,
// a Toeplitz slot likewise.
template <int NT>
struct Cfg {
  static constexpr int SA = NT == 1 ? 4 : 3;
  static constexpr int SB = NT == 1 ? 3 : 2;
  static constexpr int A_STAGE = NT * A_BYTES;  // 1 KB multiples
  static constexpr int B_STAGE = NT * B_BYTES;
  static constexpr int RINGS = SA * A_STAGE + SB * B_STAGE;
  // + 1 KB alignment slack + 256 B barriers + one generator window per X slot and term
  static constexpr size_t FIXED = (size_t)RINGS + 1024 + 256 + (size_t)SA * NT * WIN_BYTES;
};
// epilogue staging (DIR 0: transposed accumulators + operand batches; DIR 1:
// operand blocks) must fit in the pipeline stages it reuses
static_assert(8 * (2 * 32 * 33 + 3 * 16 * 32) * 4 <= Cfg<1>::RINGS, "NT=1 DIR0");
static_assert(8 * (2 * 32 * 33 + 3 * 32 * 32) * 4 <= Cfg<2>::RINGS, "NT=2 DIR0");
static_assert(8 * (3 * 32 * 32) * 4 <= Cfg<2>::RINGS, "DIR1");
static_assert(BN % 16 == 0 && BN <= ACC_COLS && 2 * ACC_COLS <= 512, "accumulator layout");
// padded generator length and the bytes of its forward + reversed copies
__host__ __device__ constexpr int gen_len(int n) { return (n + GEN_PAD + 7) / 8 * 8; }
__host__ __device__ constexpr size_t gen_bytes(int n) { return (size_t)2 * gen_len(n) * 2; }

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
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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
// bounded wait (CAP_NS, about one second in the products kernel): false on
// timeout or when another role of the CTA already gave up.  MAX_ROUNDS > 0 also
// bounds the number of polling rounds (256 polls each), independently of the
// timer.
template <uint64_t CAP_NS = 1000000000ull, uint32_t MAX_ROUNDS = 0>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  uint64_t t0 = 0;
  for (uint32_t i = 0;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255) == 255) {
      if (*abort) return false;
      const uint64_t t = global_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > CAP_NS) break;
      if (MAX_ROUNDS != 0 && (i >> 8) >= MAX_ROUNDS) break;
      __nanosleep(64);
    }
  }
  *abort = 1;
  return false;
}
// one lane per warp waits, the warp follows its verdict
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple
// of 16), completing `bytes` of the transaction count of mbarrier `bar`
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
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
// kind::f16 instruction descriptor: D F32, A/B BF16 or F16, A K-major or
// MN-major, B K-major, N = 256, M = 128
__host__ __device__ constexpr uint32_t make_idesc(bool a_mn_major, bool f16) {
  return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) |
         ((a_mn_major ? 1u : 0u) << 15) | ((uint32_t)(BN >> 3) << 17) |
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
__device__ __forceinline__ void cp_async4(float* dst_smem, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst_smem)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
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
// One job per (K block, triangle): acc 0 is the lower-Hessenberg factor
// (tile t[delta + r - k], nonzero for delta >= -256), acc 1 its transpose
// (t[-delta + k - r], nonzero for delta <= 64); delta = out0 - k0.
struct JobIter {
  int out0, kb, kb_hi;  // K blocks kb .. kb_hi - 1 (this CTA's share of the K range)
  int sub = 0;
  __device__ bool next(int& acc, int& k0, int& delta) {
    while (kb < kb_hi) {
      k0 = kb * BK;
      delta = out0 - k0;
      const int s = sub;
      if (++sub == 2) {
        sub = 0;
        ++kb;
      }
      if (s == 0 && delta >= -BN) { acc = 0; return true; }
      if (s == 1 && delta <= BK) { acc = 1; return true; }
    }
    return false;
  }
};

// first entry of the generator copy (forward | reversed, 2 glen entries) that
// row 0, column 0 of job (acc, delta) reads, and its 16-byte aligned window
__device__ __forceinline__ int job_base(int acc, int delta, int nn, int glen) {
  return acc == 0 ? glen + (nn + GEN_OFF) - delta : GEN_OFF - delta;
}
__device__ __forceinline__ int job_window(int base0) { return (base0 - 256) & ~7; }

struct KParams {
  // generator t as 16-bit copies, each [forward | reversed] of gen_len(n) entries:
  // forward f[e] = t[e - GEN_OFF], reversed r[e] = t[(n + GEN_OFF) - e], zero outside [-1, n-1]
  const uint16_t* gen_hi;
  const uint16_t* gen_lo;  // low part (split precision)
  int glen;                // gen_len of the contracted dimension
  const float* M;          // mass-term source (x-CTAs; may be null)
  float cm;
  const float *c0, *c1;    // coefficient fields of acc 0 / acc 1 (dp, dm or sigma ep, sigma em)
  float* out;
  int n1, n2;
  float inv_scale;
  int* err;
  // split K: splits > 1 CTAs (blockIdx.z) share a tile's K blocks and write
  // their partial products (coefficients applied, no mass term) to
  // ws[(DIR * splits + z) * N ..]; a reduction adds the slices in order
  int splits;
  float* ws;
};

// DIR 0: x products (rows j, columns i); DIR 1: transposed y products.
// NT: number of 16-bit terms per operand (1, or 2 for the 3-product split).
template <int DIR, int NT>
__global__ void __launch_bounds__(NUM_THREADS, 1)
toeplitz_gemm_kernel(const __grid_constant__ CUtensorMap mapA_hi,
                     const __grid_constant__ CUtensorMap mapA_lo, const KParams kp,
                     uint32_t idesc) {
  using C = Cfg<NT>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(base + C::RINGS);
  uint64_t* fullA = bars;                 // X slot filled (TMA)      [SA]
  uint64_t* emptyA = bars + C::SA;        // X slot free (MMAs done)  [SA]
  uint64_t* fullW = bars + 2 * C::SA;     // generator windows landed [SA]
  uint64_t* fullB = bars + 3 * C::SA;     // Toeplitz high term built [SB]
  // split precision: the low term of the Toeplitz operand gets its own "full"
  // barrier, so the two products that need only the high term can start
  // while the low term is still being synthesised
  uint64_t* fullL = bars + 3 * C::SA + C::SB;
  uint64_t* emptyB = bars + 3 * C::SA + 2 * C::SB;  // Toeplitz slot free [SB]
  uint64_t* accbar = bars + 3 * C::SA + 3 * C::SB;
  uint32_t* tmem_slot = (uint32_t*)(accbar + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  // generator window of X slot s, term t (WIN 16-bit entries)
  unsigned char* wins = base + C::RINGS + 256;
  auto win = [&](int s, int t) { return wins + (s * NT + t) * WIN_BYTES; };
  auto tileA = [&](int s, int t) { return base + s * C::A_STAGE + t * A_BYTES; };
  auto tileB = [&](int s, int t) {
    return base + C::SA * C::A_STAGE + s * C::B_STAGE + t * B_BYTES;
  };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // output tile: rows m0 .. m0+127 of the M dimension, columns out0 .. out0+255 of N
  const int out0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  const int nk = DIR == 0 ? (kp.n1 + BK - 1) / BK : (kp.n2 + BK - 1) / BK;
  const int kb_lo = (int)((long long)blockIdx.z * nk / kp.splits);
  const int kb_hi = (int)((long long)(blockIdx.z + 1) * nk / kp.splits);

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::SA; ++s) {
      mbar_init(smem_u32(&fullA[s]), 1);
      mbar_init(smem_u32(&emptyA[s]), 1);
      mbar_init(smem_u32(&fullW[s]), 1);
    }
    for (int s = 0; s < C::SB; ++s) {
      mbar_init(smem_u32(&fullB[s]), NSYN);
      mbar_init(smem_u32(&fullL[s]), NSYN);
      mbar_init(smem_u32(&emptyB[s]), 1);
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
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      JobIter it{out0, kb_lo, kb_hi};
      int acc, k0, delta, n = 0;
      uint32_t issued_mask = 0, parity_mask = 0;
      while (!*abort_flag && it.next(acc, k0, delta)) {
        const int s = n % C::SA;
        const uint32_t ph = (uint32_t)(n / C::SA) & 1u;
        if (!mbar_wait(smem_u32(&emptyA[s]), ph ^ 1u, abort_flag)) break;
        {
          // the generator windows this job's Toeplitz tiles are built from
          const int nn = DIR == 0 ? kp.n1 : kp.n2;
          const int ws = job_window(job_base(acc, delta, nn, kp.glen));
          const uint32_t wb = smem_u32(&fullW[s]);
          mbar_expect_tx(wb, NT * WIN_BYTES);
          for (int t = 0; t < NT; ++t)
            bulk_load(smem_u32(win(s, t)), (t == 0 ? kp.gen_hi : kp.gen_lo) + ws, WIN_BYTES, wb);
        }
        const uint32_t fb = smem_u32(&fullA[s]);
        mbar_expect_tx(fb, NT * A_BYTES);
        for (int t = 0; t < NT; ++t) {
          const CUtensorMap* map = t == 0 ? &mapA_hi : &mapA_lo;
          const uint32_t dA = smem_u32(tileA(s, t));
          if (DIR == 0) {
            tma_load_2d(dA, map, k0, m0, fb);  // X[m0.., k0..], K-major
          } else {
            tma_load_2d(dA, map, m0, k0, fb);  // X[k0.., m0..m0+63], read MN-major
            tma_load_2d(dA + A_BYTES / 2, map, m0 + 64, k0, fb);
          }
        }
        issued_mask |= 1u << s;
        parity_mask = (parity_mask & ~(1u << s)) | (ph << s);
        ++n;
      }
      const uint64_t t0 = global_ns();  // every issued copy lands before the CTA exits
      for (int s = 0; s < C::SA; ++s)
        if (issued_mask & (1u << s)) {
          while (!mbar_try(smem_u32(&fullA[s]), (parity_mask >> s) & 1u))
            if (global_ns() - t0 > 1000000000ull) break;
          while (!mbar_try(smem_u32(&fullW[s]), (parity_mask >> s) & 1u))
            if (global_ns() - t0 > 1000000000ull) break;
        }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      JobIter it{out0, kb_lo, kb_hi};
      int acc, k0, delta, n = 0;
      bool started[2] = {false, false};
      while (!*abort_flag && it.next(acc, k0, delta)) {
        const int s = n % C::SA, sb = n % C::SB;
        const uint32_t ph = (uint32_t)(n / C::SA) & 1u, phb = (uint32_t)(n / C::SB) & 1u;
        if (!mbar_wait(smem_u32(&fullA[s]), ph, abort_flag)) break;
        if (!mbar_wait(smem_u32(&fullB[sb]), phb, abort_flag)) break;
        fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * ACC_COLS);
        // (A term, B term) pairs: hi*hi and lo*hi need only the high Toeplitz
        // term; hi*lo waits for the low term
#pragma unroll
        for (int p = 0; p < (NT == 1 ? 1 : 3); ++p) {
          if (p == 2) {
            if (!mbar_wait(smem_u32(&fullL[sb]), phb, abort_flag)) break;
            fence_after();
          }
          const int ta = p == 1 ? 1 : 0, tb = p == 2 ? 1 : 0;
          const uint32_t aA = smem_u32(tileA(s, ta));
          const uint32_t aB = smem_u32(tileB(sb, tb));
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t da = DIR == 0 ? smem_desc(aA + kk * 32, 16, 1024)
                                         : smem_desc(aA + kk * 2048, A_BYTES / 2, 1024);
            const uint64_t db = smem_desc(aB + kk * 32, 16, 1024);
            mma_f16(d, da, db, idesc, (started[acc] || kk > 0 || p > 0) ? 1u : 0u);
          }
        }
        if (*abort_flag) break;
        started[acc] = true;
        mma_commit(smem_u32(&emptyA[s]));
        mma_commit(smem_u32(&emptyB[sb]));
        ++n;
      }
      mma_commit(smem_u32(accbar));  // completes when every MMA above has completed
    }
  } else {
    // ------------------------------------------------------------ synthesis
    const int w = warp - 2;  // 0..NSYN-1
    {
      // DRAM is idle while the tensor cores run: pull this warp's epilogue
      // operands (its 32 rows or columns x 128 of the tile) into L2 now, so the
      // epilogue reads them from L2 instead of waiting on DRAM
      const int g = warp & 3;
      const int c_lo = (w >> 2) ? BH : 0, c_w = (w >> 2) ? BN - BH : BH;
      auto pf = [](const float* a) { asm volatile("prefetch.global.L2 [%0];" ::"l"(a)); };
      if (DIR == 0) {
        // rows rbase + lane, this warp's columns of the tile: 128-byte lines per row
        const int row = m0 + g * 32 + lane;
        if (row < kp.n2) {
          const int c0i = out0 + c_lo;
          const int c1i = min(kp.n1, c0i + c_w) - 1;
          if (c0i <= c1i) {
            const size_t rb = (size_t)row * kp.n1;
            for (int c = c0i; c <= c1i + 31; c += 32) {
              const size_t e = rb + min(c, c1i);
              pf(kp.c0 + e);
              pf(kp.c1 + e);
              if (kp.M) pf(kp.M + e);
            }
          }
        }
      } else {
        // this warp's rows of the (transposed) tile, columns m0 + g * 32 .. + 31
        const int col = min(m0 + g * 32, kp.n1 - 1);
        for (int r = lane; r < c_w; r += 32) {
          const int row = out0 + c_lo + r;
          if (row < kp.n2) {
            const size_t e = (size_t)row * kp.n1 + col;
            pf(kp.c0 + e);
            pf(kp.c1 + e);
            pf(kp.out + e);
          }
        }
      }
    }
    {
      JobIter it{out0, kb_lo, kb_hi};
      int acc, k0, delta, n = 0;
      while (!*abort_flag && it.next(acc, k0, delta)) {
        const int s = n % C::SA, sb = n % C::SB;
        const uint32_t ph = (uint32_t)(n / C::SA) & 1u, phb = (uint32_t)(n / C::SB) & 1u;
        // the Toeplitz slot is free once the MMAs of job n - SB completed; the
        // job's generator window was prefetched with its X tiles
        if (!warp_wait(smem_u32(&emptyB[sb]), phb ^ 1u, abort_flag)) break;
        if (!warp_wait(smem_u32(&fullW[s]), ph, abort_flag)) break;
        // row r, 16-byte chunk c (k = 8c .. 8c+7) of the tile: acc 0 needs
        // t[delta + r - k] = reversed[(n + GEN_OFF) - delta - r + k], acc 1 needs
        // t[-delta + k - r] = forward[GEN_OFF - delta - r + k]: eight consecutive
        // 16-bit entries starting at e0 = base0 - r + 8c, at e0 - ws in the window
        const int nn = DIR == 0 ? kp.n1 : kp.n2;
        const int gb = job_base(acc, delta, nn, kp.glen);
        const int base0 = gb - job_window(gb);
        // A thread owns 16-byte chunk column c of an 8-row block r0 .. r0+7: row
        // r0 + u starts at entry e0 - u, e0 = base0 - r0 + 8c, so the eight chunks
        // are shifted views of entries e0 - 7 .. e0 + 7: nine words are loaded once
        // and re-aligned so that word k holds entries (e0 - 7 + 2k, e0 - 6 + 2k);
        // row u then starts 7 - u entries in -- a compile-time word and shift.
        for (int t = 0; t < NT; ++t) {
          const uint32_t* g32 = reinterpret_cast<const uint32_t*>(win(s, t));
          unsigned char* B = tileB(sb, t);
          for (int unit = w * 32 + lane; unit < (BN / 8) * 8; unit += NSYN * 32) {
            // (row block, chunk)
            const int rb = unit >> 3, c = unit & 7;
            const int r0 = rb * 8;
            const int e0 = base0 - r0 + 8 * c;
            const int wlo = (e0 - 7) >> 1;  // word holding entry e0 - 7
            const uint32_t sh0 = (uint32_t)((e0 - 7) & 1) * 16u;
            uint32_t raw[10], v[9];
#pragma unroll
            for (int k = 0; k < 10; ++k) raw[k] = g32[wlo + k];
#pragma unroll
            for (int k = 0; k < 9; ++k) v[k] = __funnelshift_r(raw[k], raw[k + 1], sh0);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int j = 7 - u;  // row u starts j entries into the window
              const int wj = j >> 1;
              uint4 chunk;
              if (j & 1) {
                chunk.x = __funnelshift_r(v[wj], v[wj + 1], 16);
                chunk.y = __funnelshift_r(v[wj + 1], v[wj + 2], 16);
                chunk.z = __funnelshift_r(v[wj + 2], v[wj + 3], 16);
                chunk.w = __funnelshift_r(v[wj + 3], v[wj + 4], 16);
              } else {
                chunk = make_uint4(v[wj], v[wj + 1], v[wj + 2], v[wj + 3]);
              }
              const int r = r0 + u;
              *reinterpret_cast<uint4*>(B + r * 128 + ((c ^ (r & 7)) << 4)) = chunk;
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the MMA
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(t == 0 ? &fullB[sb] : &fullL[sb]));
        }
        ++n;
      }
    }
    // ------------------------------------------------------------ epilogue
    const int g = warp & 3;          // TMEM lane group this warp may access
    // its part of the columns: [0, BH) or [BH, BN); the last 32-column block of
    // the upper part is partial (BN = 240)
    const int c_lo = (w >> 2) ? BH : 0, c_hi = (w >> 2) ? BN : BH;
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
      const uint32_t tl = tmem + ((uint32_t)(g * 32) << 16);
      // an accumulator none of this CTA's jobs wrote (possible with split K)
      // holds no product: it reads as zero
      float on[2] = {0.f, 0.f};
      {
        JobIter it{out0, kb_lo, kb_hi};
        int acc, k0, delta;
        while (it.next(acc, k0, delta)) on[acc] = 1.f;
      }
      const bool split = kp.splits > 1;
      float* __restrict__ wsl =
          split ? kp.ws + ((size_t)DIR * kp.splits + blockIdx.z) * ((size_t)kp.n1 * kp.n2) : nullptr;
      // The freed pipeline stages hold the epilogue's operands: each lane
      // copies its elements of a block with 4-byte cp.async (rows of a length
      // that is no multiple of 16 bytes rule out bulk copies), so all of a
      // block's loads are in flight together, and reads them back itself.
      const float* __restrict__ c0 = kp.c0;
      const float* __restrict__ c1 = kp.c1;
      float* __restrict__ out = kp.out;
      if (DIR == 0) {
        // lanes are grid rows in TMEM: stage through shared memory so lane = column
        float* stg = reinterpret_cast<float*>(base) + w * (2 * 32 * 33);
        constexpr int RB = NT == 2 ? 32 : 16;  // rows per batch of copies (fits the stages)
        float* opd = reinterpret_cast<float*>(base) + NSYN * (2 * 32 * 33) + w * (3 * RB * 32);
        const float* __restrict__ Mm = split ? nullptr : kp.M;
        float* __restrict__ dst = split ? wsl : out;
        const int rbase = m0 + g * 32;
        const int nr = kp.n2 - rbase < 32 ? kp.n2 - rbase : 32;
        for (int cb = c_lo; cb < c_hi; cb += 32) {
          const int col = out0 + cb + lane;
          const bool live = col < kp.n1 && cb + lane < BN;
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            float v[32];
            tmem_ld32(tl + a * ACC_COLS + cb, v);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 32; ++q) stg[(a * 32 + lane) * 33 + q] = on[a] * v[q];
          }
          __syncwarp();
#pragma unroll
          for (int h = 0; h < 32; h += RB) {
            if (live)
              for (int rr = 0; rr < RB && h + rr < nr; ++rr) {
                const size_t idx = (size_t)(rbase + h + rr) * kp.n1 + col;
                cp_async4(opd + (0 * RB + rr) * 32 + lane, c0 + idx);
                cp_async4(opd + (1 * RB + rr) * 32 + lane, c1 + idx);
                if (Mm) cp_async4(opd + (2 * RB + rr) * 32 + lane, Mm + idx);
              }
            cp_async_wait_all();
            if (live)
              for (int rr = 0; rr < RB && h + rr < nr; ++rr) {
                const size_t idx = (size_t)(rbase + h + rr) * kp.n1 + col;
                const float m = Mm ? opd[(2 * RB + rr) * 32 + lane] : 0.f;
                dst[idx] = kp.inv_scale * (opd[(0 * RB + rr) * 32 + lane] * stg[(h + rr) * 33 + lane] +
                                           opd[(1 * RB + rr) * 32 + lane] *
                                               stg[(32 + h + rr) * 33 + lane]) +
                           kp.cm * m;
              }
          }
          __syncwarp();
        }
      } else {
        // lanes are grid columns i; TMEM columns are grid rows j
        float* opd = reinterpret_cast<float*>(base) + w * (3 * 32 * 32);
        const int col = m0 + g * 32 + lane;
        const bool live = col < kp.n1;
        for (int cb = c_lo; cb < c_hi; cb += 32) {
          int nr = kp.n2 - (out0 + cb) < 32 ? kp.n2 - (out0 + cb) : 32;
          if (nr > BN - cb) nr = BN - cb;
          if (live)
            for (int q = 0; q < nr; ++q) {
              const size_t idx = (size_t)(out0 + cb + q) * kp.n1 + col;
              cp_async4(opd + (0 * 32 + q) * 32 + lane, c0 + idx);
              cp_async4(opd + (1 * 32 + q) * 32 + lane, c1 + idx);
              if (!split) cp_async4(opd + (2 * 32 + q) * 32 + lane, out + idx);
            }
          float a0[32], a1[32];
          tmem_ld32(tl + cb, a0);
          tmem_ld32(tl + ACC_COLS + cb, a1);
          tmem_wait_ld();
          cp_async_wait_all();
          if (live) {
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              if (q < nr) {
                const size_t idx = (size_t)(out0 + cb + q) * kp.n1 + col;
                const float prod = kp.inv_scale * (opd[(0 * 32 + q) * 32 + lane] * on[0] * a0[q] +
                                                   opd[(1 * 32 + q) * 32 + lane] * on[1] * a1[q]);
                if (split) wsl[idx] = prod;
                else out[idx] = opd[(2 * 32 + q) * 32 + lane] + prod;
              }
            }
          }
        }
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
template <typename H>
__device__ __forceinline__ float from_h(H v);
template <>
__device__ __forceinline__ float from_h<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float from_h<__half>(__half v) { return __half2float(v); }

// padded 16-bit generator copies [forward | reversed], each gen_len(n) long:
// f[e] = scale t_{e - GEN_OFF}, r[e] = scale t_{(n + GEN_OFF) - e}, zero outside
// d in [-1, n-1]; split: lo = t - hi
template <typename H>
__global__ void generator_kernel(const double* __restrict__ t, int n, float scale, H* hi, H* lo) {
  const int len = gen_len(n);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * len; e += gridDim.x * blockDim.x) {
    const int d = e < len ? e - GEN_OFF : (n + GEN_OFF) - (e - len);
    const float v = (d >= -1 && d <= n - 1) ? (float)(scale * t[d + 1]) : 0.f;
    const H h = to_h<H>(v);
    hi[e] = h;
    if (lo) lo[e] = to_h<H>(v - from_h<H>(h));
  }
}

// x (FP32, n2 x n1) -> 16-bit copies at pitch ld (hi, and lo = x - hi)
template <typename H>
__global__ void pack_kernel(const float* __restrict__ X, int n1, int n2, int ld, H* hi, H* lo) {
  const size_t N = (size_t)n1 * n2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n1), j = (int)(e / n1);
    const float v = X[e];
    const H h = to_h<H>(v);
    hi[(size_t)j * ld + i] = h;
    if (lo) lo[(size_t)j * ld + i] = to_h<H>(v - from_h<H>(h));
  }
}

// kx = cm M + sum over both directions and every split of the partial
// products, in a fixed order
__global__ void split_reduce_kernel(const float* __restrict__ ws, int splits, size_t N,
                                    const float* __restrict__ M, float cm, float* __restrict__ kx) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    float v = M ? cm * M[i] : 0.f;
    for (int q = 0; q < 2 * splits; ++q) v += ws[(size_t)q * N + i];
    kx[i] = v;
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

// Self-test of the failure path: one warp runs the bounded wait above on a
// barrier of one expected arrival.  With `complete` set, thread 0 arrives first
// and the wait succeeds; otherwise nothing arrives, the wait gives up after
// 20 ms (or 2^16 polling rounds) and the kernel raises the level's error flag
// exactly as the products kernel does.  No copy or MMA is in flight and no
// tensor memory is held, so giving up needs no draining.
constexpr uint64_t kSelftestCapNs = 20000000ull;
constexpr uint32_t kSelftestRounds = 1u << 16;

__global__ void __launch_bounds__(32) wait_selftest_kernel(int complete, int* err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (complete && threadIdx.x == 0) mbar_arrive(smem_u32(&bar));
  __syncwarp();
  int ok = 1;
  if (threadIdx.x == 0)
    ok = mbar_wait<kSelftestCapNs, kSelftestRounds>(smem_u32(&bar), 0, &abort_flag) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
}

struct Maps {
  // [term hi / lo]: x-CTAs read X K-major (box 64 x 128), y-CTAs read the
  // y-operand MN-major (box 64 x 64)
  CUtensorMap ax[2], ay[2];
  int* err;
  void *genx_hi, *genx_lo, *geny_hi, *geny_lo;
  int glen_x, glen_y;
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
  const bool split = prec == kBF16X3;
  const int nt = split ? 2 : 1;
  const size_t xbytes = (size_t)n2 * L->ld * 2;
  void** bufs[4] = {&L->xa, &L->xa_lo, &L->xb, &L->xb_lo};
  for (int b = 0; b < 4; ++b) {
    const bool need = (b % 2 == 0 || split) && (b < 2 || mass);
    if (!need) continue;
    if (cudaMalloc(bufs[b], xbytes) != cudaSuccess) return 1;
    if (cudaMemset(*bufs[b], 0, xbytes) != cudaSuccess) return 1;
  }
  Maps hm;
  std::memset(&hm, 0, sizeof(hm));
  const CUtensorMapDataType dt =
      prec == kFP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  for (int t = 0; t < nt; ++t) {
    void* xa = t == 0 ? L->xa : L->xa_lo;
    void* xb = mass ? (t == 0 ? L->xb : L->xb_lo) : xa;
    int r = encode(&hm.ax[t], dt, xa, n1, n2, (uint64_t)L->ld * 2, BK, BM);
    if (r) return r;
    r = encode(&hm.ay[t], dt, xb, n1, n2, (uint64_t)L->ld * 2, 64, BK);
    if (r) return r;
  }
  if (nt == 1) {
    hm.ax[1] = hm.ax[0];
    hm.ay[1] = hm.ay[0];
  }
  hm.glen_x = gen_len(n1);
  hm.glen_y = gen_len(n2);
  static_assert(Cfg<1>::FIXED <= 227 * 1024 && Cfg<2>::FIXED <= 227 * 1024,
                "pipeline and generator windows exceed shared memory");
  if (cudaMalloc(&hm.genx_hi, gen_bytes(n1)) != cudaSuccess) return 1;
  if (cudaMalloc(&hm.geny_hi, gen_bytes(n2)) != cudaSuccess) return 1;
  if (split) {
    if (cudaMalloc(&hm.genx_lo, gen_bytes(n1)) != cudaSuccess) return 1;
    if (cudaMalloc(&hm.geny_lo, gen_bytes(n2)) != cudaSuccess) return 1;
  }
  if (cudaMalloc(&hm.err, sizeof(int)) != cudaSuccess) return 1;
  if (cudaMemset(hm.err, 0, sizeof(int)) != cudaSuccess) return 1;
  L->maps = new Maps(hm);
  const void* kfun[4] = {(const void*)toeplitz_gemm_kernel<0, 1>,
                         (const void*)toeplitz_gemm_kernel<1, 1>,
                         (const void*)toeplitz_gemm_kernel<0, 2>,
                         (const void*)toeplitz_gemm_kernel<1, 2>};
  for (int k = 0; k < 4; ++k)
    if (cudaFuncSetAttribute(kfun[k], cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
        cudaSuccess)
      return 12;
  // split K when the tiles of a launch leave most SMs idle (e.g. n = 1023:
  // 5 x 8 tiles per direction): up to 4 CTAs per tile, each with at least
  // four K blocks
  {
    const int t0 = ((n1 + BN - 1) / BN) * ((n2 + BM - 1) / BM);
    const int t1 = ((n2 + BN - 1) / BN) * ((n1 + BM - 1) / BM);
    const int tiles = t0 > t1 ? t0 : t1;
    const int nk = ((n1 < n2 ? n1 : n2) + BK - 1) / BK;
    int sp = 152 / tiles;
    if (sp > 4) sp = 4;
    if (sp > nk / 4) sp = nk / 4;
    L->splits = sp > 1 ? sp : 1;
    if (L->splits > 1 &&
        cudaMalloc(&L->ws, (size_t)2 * L->splits * n1 * n2 * sizeof(float)) != cudaSuccess)
      return 1;
  }
  L->built = true;
  return 0;
}

int level_setup(ToeplitzGemmLevel* L, const double* tx, const double* ty, cudaStream_t st) {
  if (!L->built) return 20;
  Maps* m = (Maps*)L->maps;
  // FP16's 5-bit exponent would flush the far Toeplitz weights: scale by 2^10
  const float scale = L->prec == kFP16 ? 1024.f : 1.f;
  if (L->prec == kFP16) {
    generator_kernel<__half><<<8, 256, 0, st>>>(tx, L->n1, scale, (__half*)m->genx_hi, nullptr);
    generator_kernel<__half><<<8, 256, 0, st>>>(ty, L->n2, scale, (__half*)m->geny_hi, nullptr);
  } else {
    generator_kernel<__nv_bfloat16><<<8, 256, 0, st>>>(tx, L->n1, scale,
                                                       (__nv_bfloat16*)m->genx_hi,
                                                       (__nv_bfloat16*)m->genx_lo);
    generator_kernel<__nv_bfloat16><<<8, 256, 0, st>>>(ty, L->n2, scale,
                                                       (__nv_bfloat16*)m->geny_hi,
                                                       (__nv_bfloat16*)m->geny_lo);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : 21;
}

template <int NT>
static void launch_dir(ToeplitzGemmLevel* L, Maps* m, int dir, const float* M, double cm,
                       const float* c0, const float* c1, float* kx, bool f16, cudaStream_t st) {
  KParams kp;
  kp.cm = (float)cm;
  kp.n1 = L->n1;
  kp.n2 = L->n2;
  kp.inv_scale = f16 ? 1.f / 1024.f : 1.f;
  kp.err = m->err;
  kp.out = kx;
  kp.c0 = c0;
  kp.c1 = c1;
  kp.splits = L->splits;
  kp.ws = L->ws;
  if (dir == 0) {
    // x products: kx = cm M + dp (X A_x^T) + dm (X A_x)
    kp.M = M;
    kp.gen_hi = (const uint16_t*)m->genx_hi;
    kp.gen_lo = (const uint16_t*)(NT == 2 ? m->genx_lo : m->genx_hi);
    kp.glen = m->glen_x;
    dim3 gx((L->n1 + BN - 1) / BN, (L->n2 + BM - 1) / BM, L->splits);
    toeplitz_gemm_kernel<0, NT><<<gx, NUM_THREADS, Cfg<NT>::FIXED, st>>>(
        m->ax[0], m->ax[1], kp, make_idesc(false, f16));
  } else {
    // y products (transposed tiles): kx += ep (A_y Y) + em (A_y^T Y)
    kp.M = nullptr;
    kp.gen_hi = (const uint16_t*)m->geny_hi;
    kp.gen_lo = (const uint16_t*)(NT == 2 ? m->geny_lo : m->geny_hi);
    kp.glen = m->glen_y;
    dim3 gy((L->n2 + BN - 1) / BN, (L->n1 + BM - 1) / BM, L->splits);
    toeplitz_gemm_kernel<1, NT><<<gy, NUM_THREADS, Cfg<NT>::FIXED, st>>>(
        m->ay[0], m->ay[1], kp, make_idesc(true, f16));
  }
}

int level_pack(ToeplitzGemmLevel* L, const float* xin_x, const float* xin_y, cudaStream_t st) {
  if (!L->built) return 30;
  const int n1 = L->n1, n2 = L->n2;
  const size_t N = (size_t)n1 * n2;
  int g = (int)((N + 255) / 256);
  if (g > 152 * 16) g = 152 * 16;
  const bool two = L->xb != nullptr;
  const bool split = L->prec == kBF16X3;
  if (L->prec == kFP16) {
    pack_kernel<__half><<<g, 256, 0, st>>>(xin_x, n1, n2, L->ld, (__half*)L->xa, nullptr);
    if (two) pack_kernel<__half><<<g, 256, 0, st>>>(xin_y, n1, n2, L->ld, (__half*)L->xb, nullptr);
  } else {
    pack_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(xin_x, n1, n2, L->ld, (__nv_bfloat16*)L->xa,
                                                  (__nv_bfloat16*)(split ? L->xa_lo : nullptr));
    if (two)
      pack_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(xin_y, n1, n2, L->ld, (__nv_bfloat16*)L->xb,
                                                    (__nv_bfloat16*)(split ? L->xb_lo : nullptr));
  }
  return cudaGetLastError() == cudaSuccess ? 0 : 31;
}

int level_gemm(ToeplitzGemmLevel* L, int dir, const float* M, double cm, const float* c0,
               const float* c1, float* kx, cudaStream_t st) {
  if (!L->built) return 30;
  if (dir != 0 && dir != 1) return 32;
  Maps* m = (Maps*)L->maps;
  const bool f16 = L->prec == kFP16;
  if (L->prec == kBF16X3) launch_dir<2>(L, m, dir, M, cm, c0, c1, kx, f16, st);
  else launch_dir<1>(L, m, dir, M, cm, c0, c1, kx, f16, st);
  return cudaGetLastError() == cudaSuccess ? 0 : 31;
}

int level_finish(ToeplitzGemmLevel* L, const float* M, double cm, float* kx, cudaStream_t st) {
  if (!L->built) return 30;
  if (L->splits <= 1) return 0;
  const size_t N = (size_t)L->n1 * L->n2;
  int g = (int)((N + 255) / 256);
  if (g > 152 * 8) g = 152 * 8;
  split_reduce_kernel<<<g, 256, 0, st>>>(L->ws, L->splits, N, M, (float)cm, kx);
  return cudaGetLastError() == cudaSuccess ? 0 : 31;
}

int level_products(ToeplitzGemmLevel* L, const float* xin_x, const float* xin_y, const float* M,
                   double cm, const float* dp, const float* dm, const float* ep, const float* em,
                   float* kx, cudaStream_t st) {
  int r = level_pack(L, xin_x, xin_y, st);
  if (r) return r;
  r = level_gemm(L, 0, M, cm, dp, dm, kx, st);
  if (r) return r;
  r = level_gemm(L, 1, nullptr, 0.0, ep, em, kx, st);
  if (r) return r;
  return level_finish(L, M, cm, kx, st);
}

int level_error(ToeplitzGemmLevel* L, cudaStream_t st) {
  if (!L->built) return 0;
  Maps* m = (Maps*)L->maps;
  int e = 0;
  if (cudaMemcpyAsync(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return -1;
  if (e) cudaMemsetAsync(m->err, 0, sizeof(int), st);  // reported once
  return e;
}

int level_wait_selftest(ToeplitzGemmLevel* L, int complete, cudaStream_t st) {
  if (!L->built) return -1;
  Maps* m = (Maps*)L->maps;
  wait_selftest_kernel<<<1, 32, 0, st>>>(complete ? 1 : 0, m->err);
  return cudaGetLastError() == cudaSuccess ? 0 : 31;
}

void level_destroy(ToeplitzGemmLevel* L) {
  if (L->maps) {
    Maps* m = (Maps*)L->maps;
    cudaFree(m->err);
    cudaFree(m->genx_hi);
    cudaFree(m->genx_lo);
    cudaFree(m->geny_hi);
    cudaFree(m->geny_lo);
    delete m;
  }
  cudaFree(L->ws);
  L->ws = nullptr;
  cudaFree(L->xa);
  cudaFree(L->xa_lo);
  cudaFree(L->xb);
  cudaFree(L->xb_lo);
  L->xa = L->xa_lo = L->xb = L->xb_lo = L->maps = nullptr;
  L->built = false;
}

}  // namespace tc
}  // namespace fde
