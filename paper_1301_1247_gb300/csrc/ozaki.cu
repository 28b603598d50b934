// Complex GEMM on the 5th-generation tensor cores (tcgen05) with FP64-class accuracy, by
// splitting the operands into bf16 slices (Ozaki's error-free splitting).
//
// Each row r of op(A) is scaled by 2^-E_r (max |Re|, |Im| < 2^E_r) and each column c of B
// by 2^-E_c, and every real part is written as a 49-bit integer M = sum_i q_i 2^{7(6-i)},
// i = 0..6, with balanced digits: q_0 in [0, 128], q_1..q_6 in [-64, 64] (each one the
// rounded quotient of the remainder left by the digits before it), small integers that
// are exact in bf16.  A digit product (< 2^14) is exact in the tensor core, and
//   C_rc = 2^{E_r + E_c - 14} sum_{l=0..6} 2^{-7 l} S_l,   S_l = sum_{i+j=l} sum_k q_i q_j
// (the levels l >= 7 are dropped: together about 2^-48 of max|a| max|b| per product).  Over
// 128 values of k every |S_l| stays below 2 x 128 x (2 x 2^13 + 5 x 2^12) < 2^24, so the FP32
// accumulation in tensor memory is exact; every 128 k the seven level sums are combined in
// double-float arithmetic (FP32 pipes) into a running double-float sum per output.
//
// Per CTA: 128 x 32 outputs; tensor memory holds 7 levels x (re, im) x 32 columns of FP32
// accumulators (level l in columns 32 l and 256 + 32 l).  Shared memory is a ring of three
// stages of 16 k, each with 14 A sub-tiles (re/im x 7 digits, 128 x 16 bf16) and 14 B
// sub-tiles (32 x 16) in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes).  The
// tensor memory accelerator fills a stage with four bulk tensor copies two stages ahead of
// the MMAs: the digit planes are a 3-D tensor (k, row, plane), and a box of 8 k x all rows of
// the tile x 14 planes lands as [plane][row][8 k], i.e. one k-group of every sub-tile, core
// matrices of consecutive row groups 128 bytes apart; the two k-groups of a stage sit one
// region apart (the descriptors' leading byte offset).  Since B's digit sub-tiles follow one
// another, digit i of A meets digits 0..6-i of B in a single MMA of N = 32 (7 - i) columns
// whose result falls into the levels i..6: one thread issues the copies and 28 MMAs per
// stage (M = 128, K = 16) and commits them to the stage buffer's mbarrier; every wait is
// bounded (one second) and a timeout is reported through a status word.
#include <cuda.h>

#include <algorithm>
#include <cstdint>

#include "dense_kernels.cuh"
#include "dfcore.cuh"
#include "profile.hpp"
#include "qp_kernels.cuh"
#include "zgemm.cuh"

namespace hbs {

namespace {

constexpr int OZ_S = 7;        // digits per operand value
constexpr int OZ_BM = 128;     // rows of C per CTA (tensor-memory lanes)
constexpr int OZ_BN = 32;      // columns of C per CTA
constexpr int OZ_BK = 16;      // k per shared-memory stage (one MMA)
constexpr int OZ_FLUSH = 128;  // k per exact accumulation period
constexpr int OZ_RING = 3;     // stages in flight
constexpr int OZ_NSUB = 2 * OZ_S;                         // sub-tiles per operand and stage
constexpr int OZ_A_PL = OZ_BM * 16;                       // one plane's k-group of A: 128 rows x 16 B
constexpr int OZ_B_PL = OZ_BN * 16;                       // one plane's k-group of B: 32 rows x 16 B
constexpr int OZ_A_KG = OZ_NSUB * OZ_A_PL;                // a k-group of all 14 A planes (28 KB)
constexpr int OZ_B_KG = OZ_NSUB * OZ_B_PL;                // a k-group of all 14 B planes (7 KB)
constexpr int OZ_STAGE = 2 * (OZ_A_KG + OZ_B_KG);         // 70 KB: [A kg0 | A kg1 | B kg0 | B kg1]
constexpr int OZ_SMEM = OZ_RING * OZ_STAGE;                // 210 KB

// Exponent E with |x| < 2^E for the largest |x| given as IEEE bits (sign cleared); -2000
// for zero rows (their digits are all zero).
__device__ __forceinline__ int exp_above(unsigned long long absbits) {
  const int e = (int)(absbits >> 52);
  return e == 0 ? -2000 : e - 1022;
}

// One operand of one product: op(X) is rows x K with element (r, k) at X[r ld + k] (trans)
// or X[k ld + r]; its exponents and digit planes (14 planes of rows_pad x Kpad bf16) go to
// E and out.
struct OzOperand {
  const cplx* X;
  int ld, trans;
  int rows, K, rows_pad, Kpad;
  int* E;
  unsigned short* out;
  int nplanes;  // leading digit planes written (14; fewer when the rest are known to be zero)
};

// max(|Re|, |Im|) over each row of operand blockIdx.y: one warp per row, integer compares on
// the magnitude bits.  Rows past `rows` (padding) get the zero-row exponent.
__global__ void k_oz_exponents(const OzOperand* ops) {
  const OzOperand op = ops[blockIdx.y];
  const int lane = threadIdx.x & 31;
  for (int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); r < op.rows_pad;
       r += (int)((gridDim.x * (int64_t)blockDim.x) >> 5)) {
    unsigned long long mx = 0;
    if (r < op.rows) {
      for (int k = lane; k < op.K; k += 32) {
        const cplx v = op.trans ? op.X[(int64_t)r * op.ld + k] : op.X[(int64_t)k * op.ld + r];
        const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFull;
        const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFull;
        mx = max(mx, max(a, b));
      }
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, (unsigned long long)__shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) op.E[r] = exp_above(mx);
  }
}

// bf16 bits of the small integer (-1)^sign q (0 <= q <= 128), exact.
__device__ __forceinline__ unsigned short bf16_of_digit(unsigned int q, unsigned int sign) {
  if (q == 0u) return 0;
  const int p = 31 - __clz(q);  // q in [2^p, 2^(p+1))
  return (unsigned short)((sign << 15) | ((unsigned int)(127 + p) << 7) | ((q << (7 - p)) & 0x7Fu));
}

// The seven balanced digits of x (row exponent E) as bf16 bits, most significant first.
__device__ __forceinline__ void digits_of(double x, int E, unsigned short* out) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63);
  const int e = (int)((b >> 52) & 0x7FF);
  long long r = 0;
  if (e != 0 && E > -2000) {
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 1026 + E - e;  // |M| = round(mant 2^{e - 1075 + 49 - E}) = round(mant >> sh), sh >= 4
    if (sh < 64) r = (long long)((mant + (1ull << (sh - 1))) >> sh);
  }
#pragma unroll
  for (int i = 0; i < OZ_S - 1; ++i) {
    const int sh = 7 * (OZ_S - 1 - i);
    const long long q = (r + (1ll << (sh - 1))) >> sh;  // rounded quotient (arithmetic shift)
    r -= q * (1ll << sh);
    out[i] = bf16_of_digit((unsigned int)(q < 0 ? -q : q), sign ^ (q < 0 ? 1u : 0u));
  }
  out[OZ_S - 1] = bf16_of_digit((unsigned int)(r < 0 ? -r : r), sign ^ (r < 0 ? 1u : 0u));
}

// Digit planes of operand blockIdx.y: out[(part * 7 + d) * rows_pad * Kpad + r * Kpad + k]
// (bf16; zero beyond rows and K).
__global__ void k_oz_digits(const OzOperand* ops) {
  const OzOperand op = ops[blockIdx.y];
  const int64_t plane = (int64_t)op.rows_pad * op.Kpad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < plane; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / op.Kpad), k = (int)(e % op.Kpad);
    unsigned short dre[OZ_S], dim[OZ_S];
    if (r < op.rows && k < op.K) {
      const cplx v = op.trans ? op.X[(int64_t)r * op.ld + k] : op.X[(int64_t)k * op.ld + r];
      const int Er = op.E[r];
      digits_of(v.x, Er, dre);
      digits_of(v.y, Er, dim);
    } else {
#pragma unroll
      for (int i = 0; i < OZ_S; ++i) dre[i] = dim[i] = 0;
    }
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) {
      if (i < op.nplanes) op.out[i * plane + e] = dre[i];
      if (OZ_S + i < op.nplanes) op.out[(OZ_S + i) * plane + e] = dim[i];
    }
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: no swizzle, K-major; LBO = the byte offset between the two
// k-adjacent core matrices of a 16-k sub-tile (one k-group region), SBO = 128 B between 8-row
// groups.  The start address sits in the low 14 bits (address / 16), so the descriptor of a
// sub-tile at byte offset o from another is that descriptor plus o / 16.
__device__ __forceinline__ uint64_t oz_desc(uint32_t addr, uint32_t lbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(128 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: D f32, A and B bf16, both K-major, M = 128, N columns.
__host__ __device__ constexpr uint32_t oz_idesc(bool negA, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((negA ? 1u : 0u) << 13) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(OZ_BM >> 4) << 24);
}

__device__ __forceinline__ void oz_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// Waits for the mbarrier phase of the given parity; gives up after one second (globaltimer).
__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 1000000000ull) return false;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

// One bulk tensor copy of a box (8 k from x, rows from y, all 14 planes) of a digit-plane
// tensor into shared memory at dst, completing on the mbarrier bar.  x is a multiple of 8
// (16 bytes of bf16), as a tensor copy's innermost coordinate must be.
__device__ __forceinline__ void oz_tma_load(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(0), "r"(bar)
      : "memory");
}

// One stage (16 k from kb) of the digit planes of A (rows row0..; the first planes_a of them,
// as A's tensor map boxes hold) and of B (rows col0..) into the ring buffer at buf: announce
// the stage's bytes on its full barrier, then four copies (two k-groups of each operand).
__device__ __forceinline__ void oz_issue_stage(uint32_t buf, const CUtensorMap* tmA, const CUtensorMap* tmB, int row0,
                                               int col0, int kb, uint32_t bar, int planes_a) {
  const uint32_t bytes = 2u * (uint32_t)(planes_a * OZ_A_PL + OZ_B_KG);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  oz_tma_load(buf, tmA, kb, row0, bar);
  oz_tma_load(buf + OZ_A_KG, tmA, kb + 8, row0, bar);
  oz_tma_load(buf + 2 * OZ_A_KG, tmB, kb, col0, bar);
  oz_tma_load(buf + 2 * OZ_A_KG + OZ_B_KG, tmB, kb + 8, col0, bar);
}

// One product of a batch on the tensor cores.  Work items are (tile_m, tile_n, split);
// item_base is the prefix sum of tiles_m tiles_n splits over the earlier jobs.
struct OzJob {
  const unsigned short* Ad;  // digit planes of op(A): 14 x mpad x Kpad
  const unsigned short* Bd;  // digit planes of B^T: 14 x npad x Kpad
  const CUtensorMap* tmA;    // 3-D tensor maps of Ad and Bd (k, row, plane), boxes 8 x 128 x 14 and 8 x 32 x 14
  const CUtensorMap* tmB;
  const int* Er;
  const int* Ec;
  int m, n, mpad, npad, Kpad, klen, splits, tiles_m, tiles_n;
  int nre, nim;  // digit planes of op(A)'s real and imaginary parts that can be nonzero
  int64_t item_base;
  cplx alpha, beta;
  cplx* C;  // splits == 1: C = alpha op(A) B + beta C directly
  int ldc;
  int transC;  // C row-major
  cplx* W;  // splits > 1: alpha (partial product) per split, splits x (m x n), reduced afterwards
};

// Persistent: CTA b takes items b, b + gridDim.x, ...; tensor memory, the mbarriers and the
// shared-memory ring stay with the CTA across items (the stage counter G runs on, so every
// buffer's barrier phases are known).  Thread 0 issues the copies and the MMAs of every stage
// (warp 0 follows it stage by stage); at the end of each 128-k period all four warps meet it
// at a barrier, wait for the period's MMAs and read the accumulators.  A wait that gives up clears the CTA-wide flag s_ok, which every thread
// reads after the period's barrier, so all of them stop together.
__global__ void __launch_bounds__(128, 1) k_oz_mma(const OzJob* jobs, int njobs, int64_t nitems, int* status) {
  extern __shared__ __align__(1024) unsigned char oz_smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar[OZ_RING];   // MMAs of the buffer's stage done
  __shared__ __align__(8) uint64_t s_full[OZ_RING];  // the buffer's stage has landed
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&s_tmem)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < OZ_RING) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar[tid])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_full[tid])));
  }
  if (tid == 0) s_ok = 1;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t ring = smem_u32(oz_smem);
  const int per_flush = OZ_FLUSH / OZ_BK;
  bool ok = true;  // CTA-uniform: refreshed from s_ok after every period's barrier
  uint32_t G = 0;  // stages issued by this CTA so far

  for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].item_base <= item) lo = mid; else hi = mid - 1;
    }
    const OzJob& jb = jobs[lo];
    const int64_t local = item - jb.item_base;
    const int per = jb.tiles_m * jb.tiles_n;
    const int z = (int)(local / per), t2 = (int)(local % per);
    const int row0 = (t2 % jb.tiles_m) * OZ_BM, col0 = (t2 / jb.tiles_m) * OZ_BN;
    const int k0 = z * jb.klen, k1 = min(jb.Kpad, k0 + jb.klen);
    const int nst = (k1 - k0) / OZ_BK;
    const CUtensorMap* tmA = jb.tmA;
    const CUtensorMap* tmB = jb.tmB;
    const int planes_a = jb.nim > 0 ? OZ_NSUB : jb.nre;  // A's planes the copies bring

    float Rh[2][OZ_BN], Rl[2][OZ_BN];  // running double-float sums (re, im) of this thread's row
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int c = 0; c < OZ_BN; ++c) Rh[p][c] = Rl[p][c] = 0.f;

    bool ok0 = true;  // thread 0's own waits in this item
    if (tid == 0) {
      // the tensor maps were written by the host before the launch; order their reads by the
      // copy engine after that
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(tmA))
                   : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(tmB))
                   : "memory");
      // every earlier MMA has completed (the last period's wait covered it): all buffers are free
      oz_issue_stage(ring + (G % OZ_RING) * OZ_STAGE, tmA, tmB, row0, col0, k0, smem_u32(&s_full[G % OZ_RING]),
                     planes_a);
      if (nst > 1)
        oz_issue_stage(ring + ((G + 1) % OZ_RING) * OZ_STAGE, tmA, tmB, row0, col0, k0 + OZ_BK,
                       smem_u32(&s_full[(G + 1) % OZ_RING]), planes_a);
    }

    for (int st = 0; st < nst; ++st) {
      const uint32_t gs = G + (uint32_t)st;
      const int buf = (int)(gs % OZ_RING);
      if (warp == 0) {
        if (lane == 0 && ok0) {
          if (!oz_wait(smem_u32(&s_full[buf]), (gs / OZ_RING) & 1u)) {
            ok0 = false;
          } else {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = ring + buf * OZ_STAGE, sb = sa + 2 * OZ_A_KG;
            const uint64_t dA = oz_desc(sa, OZ_A_KG), dB = oz_desc(sb, OZ_B_KG);
            const bool fresh = (st % per_flush) == 0;
            // digit i of A against digits 0..6-i of B in one MMA: B's digit planes lie one after
            // another (32 rows each), and level l = i + j sits in columns 32 l (re) and
            // 256 + 32 l (im), so the product lands in the levels i..6 at once.
#pragma unroll
            // digits of A known to be zero (jb.nre, jb.nim) are skipped; digit 0 of the real
            // part always runs, as it opens each period's accumulators
            for (int i = 0; i < OZ_S; ++i) {
              const int N = OZ_BN * (OZ_S - i);
              const uint32_t ip = oz_idesc(false, N), in = oz_idesc(true, N);
              const uint64_t ar = dA + (uint64_t)(i * (OZ_A_PL >> 4)), ai = dA + (uint64_t)((OZ_S + i) * (OZ_A_PL >> 4));
              const uint64_t br = dB, bi = dB + (uint64_t)(OZ_S * (OZ_B_PL >> 4));
              const uint32_t dre = tmem + OZ_BN * i, dim = tmem + 256 + OZ_BN * i;
              const uint32_t first = (fresh && i == 0) ? 0u : 1u;
              if (i < jb.nre) {
                oz_mma(dre, ar, br, ip, first);  // re += Ar Br
                oz_mma(dim, ar, bi, ip, first);  // im += Ar Bi
              }
              if (i < jb.nim) {
                oz_mma(dre, ai, bi, in, 1u);  // re -= Ai Bi
                oz_mma(dim, ai, br, ip, 1u);  // im += Ai Br
              }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&s_bar[buf]))
                         : "memory");
            // refill the buffer of stage st - 1 with stage st + 2 once its MMAs are done
            if (st + 2 < nst) {
              const uint32_t pg = gs - 1;
              if (st >= 1 && !oz_wait(smem_u32(&s_bar[pg % OZ_RING]), (pg / OZ_RING) & 1u)) {
                ok0 = false;
              } else {
                const uint32_t nb = (gs + 2) % OZ_RING;
                oz_issue_stage(ring + nb * OZ_STAGE, tmA, tmB, row0, col0, k0 + (st + 2) * OZ_BK,
                               smem_u32(&s_full[nb]), planes_a);
              }
            }
          }
          if (!ok0) atomicExch(&s_ok, 0);
        }
        __syncwarp();
      }
      if ((st % per_flush) == per_flush - 1 || st == nst - 1) {
        // thread 0 arrives here only after committing this stage's MMAs, so the wait below
        // is for the buffer's current phase (a parity wait tells only two phases apart: a
        // warp running ahead of the issuing thread would see an older phase of the same
        // parity complete)
        __syncthreads();
        const bool w = oz_wait(smem_u32(&s_bar[buf]), (gs / OZ_RING) & 1u);
        if (!w) atomicExch(&s_ok, 0);
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (w) {
          // T = sum_l 2^{-7 l} S_l (Horner from l = 6), R += T, in double-float
          const uint32_t lanebase = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
          for (int p = 0; p < 2; ++p) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float th[16], tl[16], sv[16];
#pragma unroll
              for (int c = 0; c < 16; ++c) th[c] = tl[c] = 0.f;
#pragma unroll 1
              for (int l = OZ_S - 1; l >= 0; --l) {
                tmem_ld16(lanebase + 256 * p + OZ_BN * l + 16 * h, sv);
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                  th[c] *= 0.0078125f;  // 2^-7, exact
                  tl[c] *= 0.0078125f;
                  df_add_to(sv[c], 0.f, th[c], tl[c]);
                  df_norm(th[c], tl[c]);
                }
              }
#pragma unroll
              for (int c = 0; c < 16; ++c) {
                df_add_to(th[c], tl[c], Rh[p][16 * h + c], Rl[p][16 * h + c]);
                df_norm(Rh[p][16 * h + c], Rl[p][16 * h + c]);
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // tensor memory may be overwritten by the next period's MMAs
        ok = s_ok != 0;
        __syncthreads();  // every thread has read the flag before any can clear it again
        if (!ok) break;
      }
    }
    G += (uint32_t)nst;
    // ---- epilogue: this item's 128 x 32 outputs (row of this thread)
    const int row = row0 + warp * 32 + lane;
    if (row < jb.m && ok) {
      const int er = jb.Er[row];
      const cplx al = jb.alpha, be = jb.beta;
      const bool with_beta = jb.splits == 1 && (be.x != 0.0 || be.y != 0.0);
#pragma unroll
      for (int c = 0; c < OZ_BN; ++c) {
        const int col = col0 + c;
        if (col >= jb.n) break;
        const int sc = er + jb.Ec[col] - 14;
        const double re = ldexp(f2d_bits(Rh[0][c]) + f2d_bits(Rl[0][c]), sc);
        const double im = ldexp(f2d_bits(Rh[1][c]) + f2d_bits(Rl[1][c]), sc);
        cplx v = cmk(al.x * re - al.y * im, al.x * im + al.y * re);
        if (jb.splits == 1) {
          cplx* cp = jb.transC ? jb.C + (int64_t)row * jb.ldc + col : jb.C + (int64_t)col * jb.ldc + row;
          if (with_beta) v = cfma(be, *cp, v);
          *cp = v;
        } else {
          jb.W[((int64_t)z * jb.n + col) * jb.m + row] = v;
        }
      }
    }
  }
  if (!ok && tid == 0) {
    // a wait gave up: let the copies and MMAs in flight drain (bounded) before freeing
    // tensor memory and leaving the shared memory they write
    for (int b = 0; b < OZ_RING; ++b) {
      oz_wait(smem_u32(&s_full[b]), 0u);
      oz_wait(smem_u32(&s_full[b]), 1u);
      oz_wait(smem_u32(&s_bar[b]), 0u);
      oz_wait(smem_u32(&s_bar[b]), 1u);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  if (tid == 0 && !ok) atomicExch(status, 1);
}

// C = beta C + sum_s W_s (fixed order).
__global__ void k_oz_reduce(const cplx* W, int m, int n, int splits, cplx beta, cplx* C, int ldc, int transC) {
  const int64_t tot = (int64_t)m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m);
    const int64_t j = e / m;
    cplx acc = cmk(0.0, 0.0);
    for (int s = 0; s < splits; ++s) acc = cadd(acc, W[s * tot + e]);
    cplx* c = transC ? C + (int64_t)i * ldc + j : C + j * ldc + i;
    if (beta.x != 0.0 || beta.y != 0.0) acc = cfma(beta, *c, acc);
    *c = acc;
  }
}

}  // namespace

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point query, so the
// library needs no link to the driver library).
typedef CUresult (*TmapEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static TmapEncodeFn tmap_encoder() {
  static TmapEncodeFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    HBS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || p == nullptr)
      throw Error(HBS_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    return reinterpret_cast<TmapEncodeFn>(p);
  }();
  return fn;
}

// Tensor map of one operand's digit planes (14 planes of rows_pad x Kpad bf16, k contiguous)
// as a 3-D tensor (k, row, plane) with boxes of 8 k x box_rows x 14 planes.  The driver checks
// the base (16-byte aligned), the strides (multiples of 16 bytes) and the box; a failure is an
// error here, before any launch.
static void encode_planes(CUtensorMap* m, const unsigned short* base, int Kpad, int rows_pad, int box_rows,
                          int box_planes = OZ_NSUB) {
  const cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)rows_pad, (cuuint64_t)OZ_NSUB};
  const cuuint64_t strides[2] = {(cuuint64_t)Kpad * 2, (cuuint64_t)Kpad * 2 * (cuuint64_t)rows_pad};
  const cuuint32_t box[3] = {8, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = tmap_encoder()(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<unsigned short*>(base), dims,
                                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw Error(HBS_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult " + std::to_string((int)r) + ")");
}

// Products worth the tensor cores: enough k for the digit planes to pay and enough rows for
// the 128-row tiles.  (Routing the leaf products of the sweeps, k ~ 50, here as well was
// measured slower: their digit planes cost as much as the double-float product.)
bool ozaki_eligible(const GemmJob& j) { return j.k >= 96 && j.m >= 48 && j.n >= 8; }

// A batch of products on the tensor cores (see the head of this file): exponents and digit
// planes of every operand (two launches), one persistent MMA launch over all tiles, and a
// fixed-order reduction for the products split along k.
void ozaki_gemm_batched(const std::vector<GemmJob>& js, cudaStream_t s) {
  if (js.empty()) return;
  static const int sms = [] {
    int dev = 0, sm = 0;
    HBS_CUDA(cudaGetDevice(&dev));
    HBS_CUDA(cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev));
    return sm;
  }();
  static const bool attr = [] {
    HBS_CUDA(cudaFuncSetAttribute(k_oz_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    return true;
  }();
  (void)attr;
  const int nj = (int)js.size();
  std::vector<OzJob> oj(nj);
  int64_t adig = 0, bdig = 0, eA = 0, eB = 0, wtot = 0, items = 0;
  double tflops = 0.0;
  int tiles_all = 0;
  for (int q = 0; q < nj; ++q) {
    const GemmJob& j = js[q];
    OzJob& o = oj[q];
    o.m = j.m;
    o.n = j.n;
    o.tiles_m = (j.m + OZ_BM - 1) / OZ_BM;
    o.tiles_n = (j.n + OZ_BN - 1) / OZ_BN;
    o.mpad = o.tiles_m * OZ_BM;
    o.npad = o.tiles_n * OZ_BN;
    o.Kpad = (j.k + OZ_BK - 1) / OZ_BK * OZ_BK;  // stages of 16; the last period may be short
    o.nre = j.a_real_digits > 0 ? std::min(j.a_real_digits, OZ_S) : OZ_S;
    o.nim = j.a_real_digits > 0 ? 0 : OZ_S;
    tiles_all += o.tiles_m * o.tiles_n;
  }
  for (int q = 0; q < nj; ++q) {
    const GemmJob& j = js[q];
    OzJob& o = oj[q];
    // split along k only when the whole batch has too few tiles to fill the SMs
    o.splits = 1;
    if (tiles_all < sms && j.k >= 4096)
      o.splits = std::max(1, std::min(o.Kpad / OZ_FLUSH, sms / std::max(1, tiles_all)));
    o.klen = ((o.Kpad + OZ_FLUSH - 1) / OZ_FLUSH + o.splits - 1) / o.splits * OZ_FLUSH;
    o.splits = (o.Kpad + o.klen - 1) / o.klen;
    o.item_base = items;
    items += (int64_t)o.tiles_m * o.tiles_n * o.splits;
    o.alpha = j.alpha;
    o.beta = j.beta;
    o.C = j.C;
    o.ldc = j.ldc;
    o.transC = j.transC;
    o.Ad = reinterpret_cast<const unsigned short*>(adig);  // offsets for now
    o.Bd = reinterpret_cast<const unsigned short*>(bdig);
    o.Er = reinterpret_cast<const int*>(eA);
    o.Ec = reinterpret_cast<const int*>(eB);
    o.W = reinterpret_cast<cplx*>(o.splits > 1 ? wtot : 0);
    adig += (int64_t)OZ_NSUB * o.mpad * o.Kpad;
    bdig += (int64_t)OZ_NSUB * o.npad * o.Kpad;
    eA += o.mpad;
    eB += o.npad;
    if (o.splits > 1) wtot += (int64_t)o.splits * j.m * j.n;
    // executed: per digit i of A, 2 (7 - i) MMA units for its real part, 2 (7 - i) for its
    // imaginary part; 112 units in all for a general A (224 flops per m n k)
    double units = 0.0;
    for (int i = 0; i < OZ_S; ++i) units += 2.0 * (OZ_S - i) * ((i < o.nre) + (i < o.nim));
    tflops += 2.0 * units * o.mpad * (double)o.npad * o.Kpad;
  }
  DevBuf<unsigned short> Ad(adig), Bd(bdig);
  DevBuf<int> E(eA + eB), st(1);
  DevBuf<cplx> W(std::max<int64_t>(wtot, 1));
  std::vector<OzOperand> ops;
  ops.reserve(2 * nj);
  int maxrows = 0;
  int64_t maxplane = 0;
  for (int q = 0; q < nj; ++q) {
    const GemmJob& j = js[q];
    OzJob& o = oj[q];
    unsigned short* ad = Ad.get() + reinterpret_cast<int64_t>(o.Ad);
    unsigned short* bd = Bd.get() + reinterpret_cast<int64_t>(o.Bd);
    int* er = E.get() + reinterpret_cast<int64_t>(o.Er);
    int* ec = E.get() + eA + reinterpret_cast<int64_t>(o.Ec);
    // op(A) row r, k: transA ? A[r lda + k] : A[k lda + r];  B^T row c, k: B[c ldb + k]
    ops.push_back({j.A, j.lda, j.transA ? 1 : 0, j.m, j.k, o.mpad, o.Kpad, er, ad, o.nim > 0 ? OZ_NSUB : o.nre});
    ops.push_back({j.B, j.ldb, 1, j.n, j.k, o.npad, o.Kpad, ec, bd, OZ_NSUB});
    o.Ad = ad;
    o.Bd = bd;
    o.Er = er;
    o.Ec = ec;
    o.W = o.splits > 1 ? W.get() + reinterpret_cast<int64_t>(o.W) : nullptr;
    maxrows = std::max(maxrows, std::max(o.mpad, o.npad));
    maxplane = std::max(maxplane, (int64_t)std::max(o.mpad, o.npad) * o.Kpad);
  }
  HBS_CUDA(cudaMemsetAsync(st.get(), 0, sizeof(int), s));
  DevBuf<OzOperand> dops(ops.size());
  HBS_CUDA(cudaMemcpyAsync(dops.get(), ops.data(), ops.size() * sizeof(OzOperand), cudaMemcpyHostToDevice, s));
  {
    prof::KScope _ks("k_oz_digits", s);
    const unsigned bx_e = (unsigned)std::min<int64_t>(1024, ((int64_t)maxrows * 32 + 255) / 256);
    const unsigned bx_d = (unsigned)std::min<int64_t>(2048, (maxplane + 255) / 256);
    for (size_t o0 = 0; o0 < ops.size(); o0 += 65535) {
      const unsigned ny = (unsigned)std::min<size_t>(65535, ops.size() - o0);
      k_oz_exponents<<<dim3(bx_e, ny), 256, 0, s>>>(dops.get() + o0);
      k_oz_digits<<<dim3(bx_d, ny), 256, 0, s>>>(dops.get() + o0);
    }
  }
  HBS_LAUNCH_CHECK("k_oz_digits");
  // the digit planes' tensor maps, two per product, in device memory (128-byte aligned)
  std::vector<CUtensorMap> maps(2 * (size_t)nj);
  for (int q = 0; q < nj; ++q) {
    const OzJob& o = oj[q];
    encode_planes(&maps[2 * q], o.Ad, o.Kpad, o.mpad, OZ_BM, o.nim > 0 ? OZ_NSUB : o.nre);
    encode_planes(&maps[2 * q + 1], o.Bd, o.Kpad, o.npad, OZ_BN);
  }
  DevBuf<CUtensorMap> dmaps;
  dmaps.upload(maps, s);
  if (reinterpret_cast<uintptr_t>(dmaps.get()) % 128 != 0) throw Error(HBS_ERR_INTERNAL, "tensor maps misaligned");
  for (int q = 0; q < nj; ++q) {
    oj[q].tmA = dmaps.get() + 2 * q;
    oj[q].tmB = dmaps.get() + 2 * q + 1;
  }
  DevBuf<OzJob> dj(nj);
  HBS_CUDA(cudaMemcpyAsync(dj.get(), oj.data(), nj * sizeof(OzJob), cudaMemcpyHostToDevice, s));
  {
    // executed tensor work: 28 digit pairs x 4 real products x 2 flops per (padded) m n k
    prof::KScope _ks("k_oz_mma", s, tflops, 0.0);
    const unsigned grid = (unsigned)std::min<int64_t>(sms, items);
    k_oz_mma<<<grid, 128, OZ_SMEM, s>>>(dj.get(), nj, items, st.get());
  }
  HBS_LAUNCH_CHECK("k_oz_mma");
  for (int q = 0; q < nj; ++q) {
    const OzJob& o = oj[q];
    if (o.splits <= 1) continue;
    prof::KScope _ks("k_oz_reduce", s);
    k_oz_reduce<<<grid_1d((int64_t)o.m * o.n), 256, 0, s>>>(o.W, o.m, o.n, o.splits, o.beta, o.C, o.ldc, o.transC);
  }
  HBS_LAUNCH_CHECK("k_oz_reduce");
  int hs = 0;
  read_to_host(&hs, st.get(), sizeof(int), s);
  if (hs) throw Error(HBS_ERR_TIMEOUT, "tensor-core GEMM: an MMA completion wait gave up");
}

}  // namespace hbs
