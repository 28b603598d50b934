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
// accumulators (448 of the 512 columns).  Shared memory is a ring of three stages of 16 k,
// each with 14 A sub-tiles (7 digits x re/im, 128 x 16 bf16) and 14 B sub-tiles (32 x 16),
// in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes), filled by cp.async two
// stages ahead of the MMAs.  One thread issues the 112 MMAs of a stage (M = 128, N = 32,
// K = 16) and commits them to the stage buffer's mbarrier; every wait is bounded (one
// second) and a timeout is reported through a status word.
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
constexpr int OZ_A_SUB = OZ_BM * OZ_BK * 2;               // bytes of one A sub-tile (4 KB)
constexpr int OZ_B_SUB = OZ_BN * OZ_BK * 2;               // bytes of one B sub-tile (1 KB)
constexpr int OZ_STAGE = OZ_NSUB * (OZ_A_SUB + OZ_B_SUB);  // 70 KB
constexpr int OZ_SMEM = OZ_RING * OZ_STAGE;                // 210 KB

// Exponent E with |x| < 2^E for the largest |x| given as IEEE bits (sign cleared); -2000
// for zero rows (their digits are all zero).
__device__ __forceinline__ int exp_above(unsigned long long absbits) {
  const int e = (int)(absbits >> 52);
  return e == 0 ? -2000 : e - 1022;
}

// max(|Re|, |Im|) over one row of op(A) (rows = m, trans: A stored k x m) or one column of
// B (K x n, column-major): one warp per row, integer compares on the magnitude bits.
__global__ void k_oz_exponents(const cplx* X, int ld, int strided, int rows, int K, int* E) {
  const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (warp >= rows) return;
  unsigned long long mx = 0;
  for (int k = lane; k < K; k += 32) {
    const cplx v = strided ? X[(int64_t)k * ld + warp] : X[(int64_t)warp * ld + k];
    const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFull;
    mx = max(mx, max(a, b));
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, (unsigned long long)__shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) E[warp] = exp_above(mx);
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

// Digit planes of op(X) (rows x K) into out[(d * 2 + part) * rows_pad * Kpad + r * Kpad + k]
// (bf16; zero beyond rows and K).  trans = 0: element (r, k) at X[k * ld + r]; 1: X[r * ld + k].
__global__ void k_oz_digits(const cplx* X, int ld, int trans, int rows, int K, const int* E, int rows_pad, int Kpad,
                            unsigned short* out) {
  const int64_t plane = (int64_t)rows_pad * Kpad;
  const int64_t tot = plane;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / Kpad), k = (int)(e % Kpad);
    unsigned short dre[OZ_S], dim[OZ_S];
    if (r < rows && k < K) {
      const cplx v = trans ? X[(int64_t)r * ld + k] : X[(int64_t)k * ld + r];
      const int Er = E[r];
      digits_of(v.x, Er, dre);
      digits_of(v.y, Er, dim);
    } else {
#pragma unroll
      for (int i = 0; i < OZ_S; ++i) dre[i] = dim[i] = 0;
    }
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) {
      out[(2 * i) * plane + e] = dre[i];
      out[(2 * i + 1) * plane + e] = dim[i];
    }
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: no swizzle, K-major; LBO = 128 B between the two
// k-adjacent core matrices of a 16-k sub-tile, SBO = 256 B between 8-row groups.  The start
// address sits in the low 14 bits (address / 16), so the descriptor of a sub-tile at byte
// offset o from another is that descriptor plus o / 16.
__device__ __forceinline__ uint64_t oz_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: D f32, A and B bf16, both K-major, M = 128, N = 32.
__host__ __device__ constexpr uint32_t oz_idesc(bool negA) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((negA ? 1u : 0u) << 13) | ((uint32_t)(OZ_BN >> 3) << 17) |
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

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// One stage (16 k from kb) of every digit plane into ring buffer `buf`: 16-byte chunks
// (8 bf16 along k) into the core-matrix layout [row group][k group][8 rows][16 B].
__device__ __forceinline__ void oz_load_stage(unsigned char* buf, const unsigned short* Ad, const unsigned short* Bd,
                                              int64_t aplane, int64_t bplane, int Kpad, int row0, int col0, int kb,
                                              int tid) {
  for (int q = tid; q < OZ_NSUB * OZ_BM * 2; q += 128) {
    const int sub = q / (OZ_BM * 2), rem = q % (OZ_BM * 2), r = rem >> 1, c8 = rem & 1;
    const unsigned short* src = Ad + sub * aplane + (int64_t)(row0 + r) * Kpad + kb + 8 * c8;
    cp_async16(smem_u32(buf + sub * OZ_A_SUB + ((r >> 3) * 2 + c8) * 128 + (r & 7) * 16), src);
  }
  unsigned char* bb = buf + OZ_NSUB * OZ_A_SUB;
  for (int q = tid; q < OZ_NSUB * OZ_BN * 2; q += 128) {
    const int sub = q / (OZ_BN * 2), rem = q % (OZ_BN * 2), r = rem >> 1, c8 = rem & 1;
    const unsigned short* src = Bd + sub * bplane + (int64_t)(col0 + r) * Kpad + kb + 8 * c8;
    cp_async16(smem_u32(bb + sub * OZ_B_SUB + ((r >> 3) * 2 + c8) * 128 + (r & 7) * 16), src);
  }
}

// grid (tiles_m, tiles_n, splits).  Ad: digit planes of op(A) (mpad x Kpad), Bd: of B^T
// (npad x Kpad).  Split z covers k in [z klen, (z + 1) klen) (klen a multiple of 128).
// W: m x n (ld m) per split, alpha 2^{E_r + E_c - 14} sum_l 2^{-7 l} S_l in FP64.
__global__ void __launch_bounds__(128, 1) k_oz_mma(const unsigned short* Ad, const unsigned short* Bd, int mpad,
                                                    int npad, int Kpad, int klen, const int* Er, const int* Ec,
                                                    int m, int n, cplx alpha, cplx* W, int* status) {
  extern __shared__ __align__(1024) unsigned char oz_smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar[OZ_RING];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * OZ_BM, col0 = blockIdx.y * OZ_BN;
  const int k0 = blockIdx.z * klen, k1 = min(Kpad, k0 + klen);
  const int nst = (k1 - k0) / OZ_BK;
  const int64_t aplane = (int64_t)mpad * Kpad, bplane = (int64_t)npad * Kpad;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&s_tmem)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < OZ_RING) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar[tid])));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  float Rh[2][OZ_BN], Rl[2][OZ_BN];  // running double-float sums (re, im) of this thread's row
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int c = 0; c < OZ_BN; ++c) Rh[p][c] = Rl[p][c] = 0.f;

  // prologue: stages 0 and 1 in flight
  oz_load_stage(oz_smem, Ad, Bd, aplane, bplane, Kpad, row0, col0, k0, tid);
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (nst > 1) oz_load_stage(oz_smem + OZ_STAGE, Ad, Bd, aplane, bplane, Kpad, row0, col0, k0 + OZ_BK, tid);
  asm volatile("cp.async.commit_group;" ::: "memory");

  bool ok = true;
  const int per_flush = OZ_FLUSH / OZ_BK;
  for (int st = 0; st < nst && ok; ++st) {
    const int buf = st % OZ_RING;
    unsigned char* sbuf = oz_smem + buf * OZ_STAGE;
    asm volatile("cp.async.wait_group 1;" ::: "memory");  // stage st has landed (st + 1 may be in flight)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ip = oz_idesc(false), in = oz_idesc(true);
      const uint64_t dA = oz_desc(smem_u32(sbuf)), dB = oz_desc(smem_u32(sbuf + OZ_NSUB * OZ_A_SUB));
      const bool fresh = (st % per_flush) == 0;
#pragma unroll
      for (int l = 0; l < OZ_S; ++l) {
        const uint32_t dre = tmem + 64 * l, dim = dre + 32;
#pragma unroll
        for (int i = 0; i <= l; ++i) {
          const int j = l - i;
          const uint64_t ar = dA + (uint64_t)((2 * i) * (OZ_A_SUB >> 4)), ai = ar + (OZ_A_SUB >> 4);
          const uint64_t br = dB + (uint64_t)((2 * j) * (OZ_B_SUB >> 4)), bi = br + (OZ_B_SUB >> 4);
          const uint32_t first = (fresh && i == 0) ? 0u : 1u;
          oz_mma(dre, ar, br, ip, first);  // re += Ar Br
          oz_mma(dre, ai, bi, in, 1u);     // re -= Ai Bi
          oz_mma(dim, ar, bi, ip, first);  // im += Ar Bi
          oz_mma(dim, ai, br, ip, 1u);     // im += Ai Br
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&s_bar[buf]))
                   : "memory");
    }
    __syncwarp();
    // refill the buffer of stage st - 1 with stage st + 2 once its MMAs are done
    if (st + 2 < nst) {
      if (st >= 1) {
        const int pb = (st - 1) % OZ_RING;
        if (!oz_wait(smem_u32(&s_bar[pb]), (uint32_t)(((st - 1) / OZ_RING) & 1))) ok = false;
      }
      oz_load_stage(oz_smem + ((st + 2) % OZ_RING) * OZ_STAGE, Ad, Bd, aplane, bplane, Kpad, row0, col0,
                    k0 + (st + 2) * OZ_BK, tid);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");  // possibly empty: keeps the group count uniform
    if ((st % per_flush) == per_flush - 1 || st == nst - 1) {
      if (!oz_wait(smem_u32(&s_bar[buf]), (uint32_t)((st / OZ_RING) & 1))) ok = false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (ok) {
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
              tmem_ld16(lanebase + 64 * l + 32 * p + 16 * h, sv);
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
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // ---- epilogue: scale and store this split's partial result
  const int row = row0 + warp * 32 + lane;
  if (row < m && ok) {
    const int er = Er[row];
#pragma unroll
    for (int c = 0; c < OZ_BN; ++c) {
      const int col = col0 + c;
      if (col >= n) break;
      const int sc = er + Ec[col] - 14;
      const double re = ldexp(f2d_bits(Rh[0][c]) + f2d_bits(Rl[0][c]), sc);
      const double im = ldexp(f2d_bits(Rh[1][c]) + f2d_bits(Rl[1][c]), sc);
      W[((int64_t)blockIdx.z * n + col) * m + row] = cmk(alpha.x * re - alpha.y * im, alpha.x * im + alpha.y * re);
    }
  }
  if (!ok) {  // a wait gave up: let the MMAs in flight drain (bounded) before freeing tensor memory
    for (int b = 0; b < OZ_RING; ++b) {
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
__global__ void k_oz_reduce(const cplx* W, int m, int n, int splits, cplx beta, cplx* C, int ldc) {
  const int64_t tot = (int64_t)m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m);
    const int64_t j = e / m;
    cplx acc = cmk(0.0, 0.0);
    for (int s = 0; s < splits; ++s) acc = cadd(acc, W[s * tot + e]);
    cplx* c = C + j * ldc + i;
    if (beta.x != 0.0 || beta.y != 0.0) acc = cfma(beta, *c, acc);
    *c = acc;
  }
}

}  // namespace

bool ozaki_eligible(const GemmJob& j) { return j.k >= 4096 && j.m >= 64 && j.n >= 16; }

// One GEMM job on the tensor cores (see the head of this file).
void ozaki_gemm(const GemmJob& j, cudaStream_t s) {
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
  const int m = j.m, n = j.n, K = j.k;
  const int tm = (m + OZ_BM - 1) / OZ_BM, tn = (n + OZ_BN - 1) / OZ_BN;
  const int mpad = tm * OZ_BM, npad = tn * OZ_BN;
  const int Kpad = (K + OZ_FLUSH - 1) / OZ_FLUSH * OZ_FLUSH;
  // one wave: at most one CTA per SM (each holds all of tensor memory)
  int splits = std::max(1, std::min(Kpad / OZ_FLUSH, sms / (tm * tn)));
  int klen = (Kpad / OZ_FLUSH + splits - 1) / splits * OZ_FLUSH;
  splits = (Kpad + klen - 1) / klen;
  DevBuf<int> Er(mpad), Ec(npad), st(1);
  DevBuf<unsigned short> Ad((size_t)OZ_NSUB * mpad * Kpad), Bd((size_t)OZ_NSUB * npad * Kpad);
  DevBuf<cplx> W((size_t)splits * m * n);
  HBS_CUDA(cudaMemsetAsync(st.get(), 0, sizeof(int), s));
  {
    prof::KScope _ks("k_oz_digits", s);
    // op(A) row r, k: transA ? A[r lda + k] : A[k lda + r];  B^T row c, k: B[c ldb + k]
    k_oz_exponents<<<(m * 32 + 255) / 256, 256, 0, s>>>(j.A, j.lda, j.transA ? 0 : 1, m, K, Er.get());
    k_oz_exponents<<<(n * 32 + 255) / 256, 256, 0, s>>>(j.B, j.ldb, 0, n, K, Ec.get());
    k_oz_digits<<<grid_1d((int64_t)mpad * Kpad), 256, 0, s>>>(j.A, j.lda, j.transA ? 1 : 0, m, K, Er.get(), mpad,
                                                              Kpad, Ad.get());
    k_oz_digits<<<grid_1d((int64_t)npad * Kpad), 256, 0, s>>>(j.B, j.ldb, 1, n, K, Ec.get(), npad, Kpad, Bd.get());
  }
  HBS_LAUNCH_CHECK("k_oz_digits");
  {
    // executed tensor work: 28 digit pairs x 4 real products x 2 flops per (padded) m n k
    prof::KScope _ks("k_oz_mma", s, 224.0 * mpad * (double)npad * Kpad, 0.0);
    k_oz_mma<<<dim3(tm, tn, splits), 128, OZ_SMEM, s>>>(Ad.get(), Bd.get(), mpad, npad, Kpad, klen, Er.get(),
                                                         Ec.get(), m, n, j.alpha, W.get(), st.get());
  }
  HBS_LAUNCH_CHECK("k_oz_mma");
  {
    prof::KScope _ks("k_oz_reduce", s);
    k_oz_reduce<<<grid_1d((int64_t)m * n), 256, 0, s>>>(W.get(), m, n, splits, j.beta, j.C, j.ldc);
  }
  HBS_LAUNCH_CHECK("k_oz_reduce");
  int hs = 0;
  HBS_CUDA(cudaMemcpyAsync(&hs, st.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  HBS_CUDA(cudaStreamSynchronize(s));
  if (hs) throw Error(HBS_ERR_TIMEOUT, "tensor-core GEMM: an MMA completion wait gave up");
}

}  // namespace hbs
