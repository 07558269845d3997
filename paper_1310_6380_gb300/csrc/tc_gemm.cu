// Exact-slice contractions on the tcgen05 tensor cores.
//
// D[z][n][m] = sum_k A[z][m][k] B[z][n][k] for BF16 A (M x K) and B (N x K),
// both K-contiguous, with FP32 accumulation in tensor memory and FP32 D
// stored n-major (column-major M x N).  One CTA computes a 128 x BN tile:
// a TMA producer thread streams 128 x 64 tiles of A and BN x 64 tiles of B
// through a 3-stage shared-memory ring (128-byte swizzle, mbarrier
// completion), one thread issues tcgen05.mma (kind::f16, M=128, N=BN, K=16)
// into a TMEM accumulator, and all four warps drain TMEM with tcgen05.ld.
// The ring is sized so that two CTAs fit on an SM: one drains its
// accumulator while the other's MMAs run.  BN (64..128, a multiple of 16)
// is chosen per launch: the largest that pads N by at most 6 %.
//
// The library feeds it "digit planes": an FP64 operand x with per-row
// scale 2^e is written as sum_s t_s 2^(e - 6 - 7s) with integer digits
// |t_s| <= 64 (balanced rounding, radix 2^7).  Every product of two digits
// is an integer of magnitude <= 2^12 and every sum over at most 4032 terms
// stays below 2^24, so the FP32 accumulation is exact.  The S digit planes
// sit side by side along K (B's in reverse order), so one slab of the
// contraction forms a whole digit order sum_{s+t=u} A_s B_t^T at once; the
// slab table (order, first A and B column, length) rides in the kernel's
// parameters and blockIdx.z picks the slab.  The FP64 recombination of the
// orders u < S reproduces the FP64 contraction to about 2^-46 of |A||B|
// (seven digits) on the BF16 tensor pipe.
#include <atomic>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "bs_internal.h"

namespace {

constexpr int BM = 128, BK = 64, STAGES = 3;
constexpr int TILE_A = BM * BK * 2;                    // bytes per stage
__host__ __device__ constexpr int tile_b(int bn) { return bn * BK * 2; }
__host__ __device__ constexpr int smem_bytes(int bn) { return STAGES * (TILE_A + tile_b(bn)) + 1024; }
constexpr int TMEM_COLS = 128;                         // power of two >= BN
constexpr long WAIT_LIMIT = 1L << 20;   // try_wait rounds before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: sets *err and returns false when the phase never completes
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  for (long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicOr(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;              // leading-dimension offset (unused when swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride-dimension offset
  d |= (uint64_t)1 << 46;              // descriptor version of tcgen05
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// instruction descriptor, kind::f16: D f32, A bf16, B bf16, both K-major
__host__ __device__ constexpr uint32_t idesc(int bn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

// blockIdx.z = z * slabs.nq + q: batch entry z, slab q (one slab of the
// whole K for a plain contraction)
template <int BN>
__global__ void __launch_bounds__(128, 2)
    slice_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, float* __restrict__ D, int M,
                      int N, long ldd, long strideD, const SliceSlabs slabs,
                      int* __restrict__ err) {
  constexpr int TILE_B = tile_b(BN);
  constexpr uint32_t IDESC = idesc(BN);
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_base;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * TILE_A;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.z % slabs.nq, z = blockIdx.z / slabs.nq;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int ka = slabs.a0[q], kbb = slabs.b0[q];
  const int nk = (slabs.len[q] + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (kb >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, err)) break;
      mbar_expect_tx(&full[s], TILE_A + TILE_B);
      tma_load_3d(sA + s * TILE_A, &tmA, ka + kb * BK, m0, z, &full[s]);
      tma_load_3d(sB + s * TILE_B, &tmB, kbb + kb * BK, n0, z, &full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(&full[s], ph, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA + s * TILE_A), b0 = smem_u32(sB + s * TILE_B);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t ad = sdesc(a0 + kk * 32), bd = sdesc(b0 + kk * 32);
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&empty[s]))
          : "memory");
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&done))
        : "memory");
  }
  __syncwarp();
  // tcgen05.ld is warp-collective: every lane of a warp takes the same branch
  const bool ok = __all_sync(0xffffffffu, mbar_wait(&done, 0u, err));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int m = m0 + warp * 32 + lane;
    float* dz = D + (size_t)blockIdx.z * strideD;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t v[16];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          if (n < N) dz[(size_t)n * ldd + m] = __uint_as_float(v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

// ---- fused rank-2nb update of the dense-to-band reduction (band.cu):
// A22 -= X Y^dagger with X = [V W], Y = [W V] given as eight digit planes
// per operand (slices.cu, pack_rank2_kernel): A rows r [A_0 | .. | A_7],
// B rows (c, part) reversed [B_7 | .. | B_0], each block 64 wide.  The CTA
// keeps all eight digit orders u = s + t of its 128 x BN tile in tensor
// memory (accumulator u at column u BN), streams A's digit blocks through
// a ring while B's stay resident, and the epilogue combines the orders in
// a 64-bit integer and subtracts the product from the FP64 matrix in place,
// so no partial products go through global memory.  The update is
// Hermitian: tiles above the diagonal exit at once, and the others write
// A22[r, c] (r >= c) and, staged through shared memory so that the stores
// run along columns, A22[c, r] = conj(A22[r, c]).
//
// Order sums: with at most 64 nonzero terms per digit block (K = 4 nb),
// |o_u| <= (u + 1) 2^18, so hi = sum_{u<4} o_u 2^(7(3-u)) < 2^40 and
// T = hi 2^21 + floor(lo / 2^7), lo = sum_{u>=4} o_u 2^(7(7-u)), is below
// 2^62: sum_u 2^(-12-7u) o_u = 2^-54 T up to 2^-54 of the operands' scale,
// the size of the digit truncation itself.  One conversion and one FMA per
// real entry (GB300 issues 2 FP64 operations per clock per SM).
constexpr int R2_S = 8;

template <int BN, int R2_STAGES, int MINB, int NT>
__global__ void __launch_bounds__(NT, MINB)
    rank2_update_kernel(const __grid_constant__ CUtensorMap tmA,
                        const __grid_constant__ CUtensorMap tmB, const int* __restrict__ ex,
                        int m, zd* __restrict__ A, int n, int o, int ct0,
                        int* __restrict__ err) {
  constexpr int TILE_B = tile_b(BN);
  constexpr uint32_t IDESC = idesc(BN);
  constexpr int TCOLS = R2_S * BN;   // 256 or 512
  constexpr int CW = BN / 2;         // complex columns of the tile
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[R2_STAGES], empty[R2_STAGES], bfull, done;
  __shared__ uint32_t tmem_base;
  const int z = blockIdx.z;
  const int m0 = blockIdx.x * BM, n0 = (blockIdx.y + ct0) * BN, cc0 = n0 / 2;
  if (cc0 > m0 + BM - 1) return;     // above the diagonal: the mirror tile writes it
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + R2_STAGES * TILE_A;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int q = 0; q < R2_STAGES; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    mbar_init(&bfull, 1);
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // TMA producer: B's eight blocks once, then A's digit blocks through the ring
    mbar_expect_tx(&bfull, R2_S * TILE_B);
    for (int b = 0; b < R2_S; ++b) tma_load_3d(sB + b * TILE_B, &tmB, b * BK, n0, z, &bfull);
    for (int sd = 0; sd < R2_S; ++sd) {
      const int q = sd % R2_STAGES;
      const uint32_t ph = (uint32_t)(sd / R2_STAGES) & 1u;
      if (sd >= R2_STAGES && !mbar_wait(&empty[q], ph ^ 1u, err)) break;
      mbar_expect_tx(&full[q], TILE_A);
      tma_load_3d(sA + q * TILE_A, &tmA, sd * BK, m0, z, &full[q]);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: digit s of A against digits t = 0 .. 7-s of B into order s + t
    bool ok = mbar_wait(&bfull, 0u, err);
    for (int sd = 0; ok && sd < R2_S; ++sd) {
      const int q = sd % R2_STAGES;
      const uint32_t ph = (uint32_t)(sd / R2_STAGES) & 1u;
      if (!mbar_wait(&full[q], ph, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA + q * TILE_A);
      for (int t = 0; t + sd < R2_S; ++t) {
        const uint32_t b0 = smem_u32(sB + (R2_S - 1 - t) * TILE_B);
        const uint32_t acc_addr = tmem + (uint32_t)((sd + t) * BN);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t ad = sdesc(a0 + kk * 32), bd = sdesc(b0 + kk * 32);
          const uint32_t acc = (sd > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc_addr),
              "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&empty[q]))
          : "memory");
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&done))
        : "memory");
  }
  __syncwarp();
  // The epilogue: warps w and w + 4 share the TMEM lanes (rows) of quadrant
  // w % 4 and take half of the tile's columns each.  While TMA and the MMAs
  // run, every thread fetches the FP64 entries of its row and columns that
  // the tile updates (the epilogue is otherwise bound by these loads' DRAM
  // latency).
  constexpr int HALVES = NT / 128, CWH = CW / HALVES, BNH = BN / HALVES;
  const int quad = warp & 3, half = warp >> 2;
  const int rl = quad * 32 + lane, r = m0 + rl;
  const bool live = r < m;
  zd* az = A + (size_t)z * n * n + (size_t)o * n + o;
  zd old[CWH];
  int ec[CWH];
#pragma unroll
  for (int h = 0; h < CWH; ++h) {
    const int c = cc0 + half * CWH + h;
    const bool use = live && c < m && c <= r;
    old[h] = use ? az[(size_t)c * n + r] : zmake(0.0, 0.0);
    ec[h] = c < m ? ex[(size_t)z * m + c] : 0;
  }
  const int er = live ? ex[(size_t)z * m + r] : 0;
  const bool ok = __all_sync(0xffffffffu, mbar_wait(&done, 0u, err));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // the A ring is free once every MMA has completed: it stages the tile
  // (BM x CW complex, row stride CW + 1) for the transposed stores
  zd* stage = reinterpret_cast<zd*>(sA);
  if (ok) {
    // four columns (two complex) at a time: the eight digit orders' loads
    // are issued together and waited for once
#pragma unroll
    for (int cq = 0; cq < BNH; cq += 4) {
      const int c0 = half * BNH + cq;
      uint32_t v[R2_S][4];
#pragma unroll
      for (int u = 0; u < R2_S; ++u) {
        const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(u * BN + c0);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v[u][0]), "=r"(v[u][1]), "=r"(v[u][2]), "=r"(v[u][3])
                     : "r"(ta));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      long long hi[4], lo[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        // the order sums are exact integers below 2^22: the FP32 add of
        // 1.5 2^23 puts them in the low mantissa bits; pairs of orders
        // o_u 2^7 + o_{u+1} stay below 2^29 and combine in 32 bits
        int d[R2_S];
#pragma unroll
        for (int u = 0; u < R2_S; ++u)
          d[u] = __float_as_int(__uint_as_float(v[u][jj]) + 12582912.0f) - 0x4B400000;
        const int p0 = d[0] * 128 + d[1], p1 = d[2] * 128 + d[3];
        const int p2 = d[4] * 128 + d[5], p3 = d[6] * 128 + d[7];
        hi[jj] = (long long)p0 * 16384 + p1;
        lo[jj] = (long long)p2 * 16384 + p3;
      }
#pragma unroll
      for (int jc = 0; jc < 2; ++jc) {
        const int h = cq / 2 + jc, cl = half * CWH + h, c = cc0 + cl;
        zd val = zmake(0.0, 0.0);
        if (live && c < m && c <= r) {
          const long long tr = hi[2 * jc] * 2097152 + (lo[2 * jc] >> 7);
          const long long ti = hi[2 * jc + 1] * 2097152 + (lo[2 * jc + 1] >> 7);
          const double w = __longlong_as_double((long long)(1023 + er + ec[h] - 54) << 52);
          val = old[h];
          val.x = fma(-(double)tr, w, val.x);
          val.y = r == c ? 0.0 : fma(-(double)ti, w, val.y);
          az[(size_t)c * n + r] = val;
        }
        stage[rl * (CW + 1) + cl] = val;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TCOLS));
  }
  if (ok) {
    // A22[c, r] = conj(A22[r, c]) for r > c: CW consecutive c per row r
    for (int idx = threadIdx.x; idx < BM * CW; idx += NT) {
      const int rr = idx / CW, cl = idx % CW;
      const int rw = m0 + rr, c = cc0 + cl;
      if (rw < m && c < m && rw > c) az[(size_t)rw * n + c] = zconj(stage[rr * (CW + 1) + cl]);
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

int make_map(CUtensorMap* tm, const uint16_t* base, int K, int rows, int batch, long bstride,
             int box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    bs_set_error("cuTensorMapEncodeTiled is unavailable");
    return BS_ECUDA;
  }
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)K * 2, (cuuint64_t)bstride * 2};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    bs_set_error("cuTensorMapEncodeTiled failed (%d): K=%d rows=%d batch=%d", (int)r, K, rows,
                 batch);
    return BS_ECUDA;
  }
  return BS_OK;
}

// the tile edge along N: the largest candidate that pads N by at most 6 %
// (larger tiles read each A tile fewer times and issue larger MMAs), else
// the one that pads least
static int pick_bn(int N) {
  static const int cand[] = {128, 112, 96, 80, 64};
  for (int bn : cand)
    if ((long)((N + bn - 1) / bn) * bn - N <= 0.06 * N) return bn;
  int best = 128;
  long waste = -1;
  for (int bn : cand) {
    const long w = (long)((N + bn - 1) / bn) * bn - N;
    if (waste < 0 || w < waste) {
      waste = w;
      best = bn;
    }
  }
  return best;
}

template <int BN>
static int launch_bn(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int K,
                     int batch, long sA, long sB, long ldd, long sD, const SliceSlabs& slabs,
                     int* err, cudaStream_t s) {
  CUtensorMap ta, tb;
  int r = make_map(&ta, A, K, M, batch, sA, BM);
  if (!r) r = make_map(&tb, B, K, N, batch, sB, BN);
  if (r) return r;
  // the shared-memory opt-in is a per-device attribute of the kernel
  static std::atomic<bool> attr[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (!attr[dev].load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(slice_gemm_kernel<BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes(BN));
    if (e != cudaSuccess) return bs_cuda_status(e, "slice GEMM smem");
    attr[dev].store(true, std::memory_order_release);
  }
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN, batch * slabs.nq);
  slice_gemm_kernel<BN><<<grid, 128, smem_bytes(BN), s>>>(ta, tb, D, M, N, ldd, sD, slabs, err);
  BS_CHECK_LAUNCH("slice_gemm_kernel");
  return BS_OK;
}

static int dispatch_bn(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int K,
                       int batch, long sA, long sB, long ldd, long sD, const SliceSlabs& slabs,
                       int* err, cudaStream_t s) {
  switch (pick_bn(N)) {
    case 64: return launch_bn<64>(A, B, D, M, N, K, batch, sA, sB, ldd, sD, slabs, err, s);
    case 80: return launch_bn<80>(A, B, D, M, N, K, batch, sA, sB, ldd, sD, slabs, err, s);
    case 96: return launch_bn<96>(A, B, D, M, N, K, batch, sA, sB, ldd, sD, slabs, err, s);
    case 112: return launch_bn<112>(A, B, D, M, N, K, batch, sA, sB, ldd, sD, slabs, err, s);
    default: return launch_bn<128>(A, B, D, M, N, K, batch, sA, sB, ldd, sD, slabs, err, s);
  }
}

}  // namespace

// slabs of at most L terms (L % 64 == 0); false when there are more than BS_SLAB_MAX
static bool cut_slabs(int S, int Kp, int L, SliceSlabs* sl) {
  sl->nq = 0;
  for (int u = 0; u < S; ++u) {
    const int len = (u + 1) * Kp;
    for (int k0 = 0; k0 < len; k0 += L) {
      if (sl->nq == BS_SLAB_MAX) return false;
      const int q = sl->nq++;
      sl->order[q] = u;
      sl->a0[q] = k0;
      sl->b0[q] = (S - 1 - u) * Kp + k0;
      sl->len[q] = len - k0 < L ? len - k0 : L;
    }
  }
  return true;
}

// The longest slabs (fewest FP32 partial products to store and add) unless
// the launch would then leave SMs idle: while the CTAs number fewer than two
// per SM, the slabs are halved (down to 128 terms), which trades a serial K
// loop for parallel CTAs.  Small contractions (one cell's form factors) need
// this; batched ones keep the longest slabs.
bool bs_slice_slabs(int S, int Kp, int M, int N, int batch, SliceSlabs* sl) {
  const int bn = pick_bn(N);
  const long tiles = (long)((M + BM - 1) / BM) * ((N + bn - 1) / bn) * batch;
  const long want = 2L * bs_sm_count();
  int L = BS_SLAB_K;
  if (!cut_slabs(S, Kp, L, sl)) return false;
  while (tiles * sl->nq < want && L > 128) {
    const int L2 = (L / 2) / 64 * 64 < 128 ? 128 : (L / 2) / 64 * 64;
    SliceSlabs t;
    if (!cut_slabs(S, Kp, L2, &t)) break;
    *sl = t;
    L = L2;
  }
  return true;
}

size_t bs_slice_planes(int S, int Kp, int M, int N, int batch) {
  // a smaller batch may cut its slabs finer: take the largest count of
  // (entry, slab) output planes over every batch size up to `batch`
  SliceSlabs full, sl;
  if (!cut_slabs(S, Kp, BS_SLAB_K, &full)) return (size_t)BS_SLAB_MAX * batch;
  const int bn = pick_bn(N);
  const long t1 = (long)((M + BM - 1) / BM) * ((N + bn - 1) / bn);
  size_t best = (size_t)full.nq * batch;
  // from the first batch size whose longest slabs already give two CTAs per
  // SM on, nothing is cut and the count grows with the batch
  for (int b = 1; b <= batch && t1 * full.nq * b < 2L * bs_sm_count(); ++b) {
    if (!bs_slice_slabs(S, Kp, M, N, b, &sl)) return (size_t)BS_SLAB_MAX * batch;
    const size_t v = (size_t)sl.nq * b;
    if (v > best) best = v;
  }
  return best;
}

int bs_launch_slice_gemm(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int K,
                         int batch, long sA, long sB, long ldd, long sD, int* err,
                         cudaStream_t s) {
  if (K % 8 != 0 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || sA % 8 || sB % 8 || K > 4096 ||
      M < 1 || N < 1 || batch < 1 || batch > 65535) {
    bs_set_error("slice GEMM: need K %% 8 == 0, K <= 4096, 16-byte aligned operands");
    return BS_EINVAL;
  }
  SliceSlabs one;
  one.nq = 1;
  one.order[0] = 0;
  one.a0[0] = one.b0[0] = 0;
  one.len[0] = K;
  return dispatch_bn(A, B, D, M, N, K, batch, sA, sB, ldd, sD, one, err, s);
}

int bs_launch_slice_orders(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int S,
                           int Kp, int batch, int* err, cudaStream_t s) {
  SliceSlabs sl;
  if (Kp % 64 != 0 || S < 1 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || M < 1 || N < 1 ||
      batch < 1 || !bs_slice_slabs(S, Kp, M, N, batch, &sl) || (long)batch * sl.nq > 65535) {
    bs_set_error("slice orders: need Kp %% 64 == 0, 16-byte aligned operands, at most %d slabs",
                 BS_SLAB_MAX);
    return BS_EINVAL;
  }
  const int K = S * Kp;
  return dispatch_bn(A, B, D, M, N, K, batch, (long)M * K, (long)N * K, M, (long)M * N, sl, err,
                     s);
}

// A22 (m x m at offset o of each n x n matrix) -= X Y^dagger from the digit
// planes of pack_rank2_kernel; ex: row exponents (kb x m)
int bs_rank2_column_tiles(int m) { return (2 * m + 31) / 32; }

// column tiles ct0 .. ct0 + nct - 1 (16 complex columns each; nct <= 0: to the end)
int bs_launch_rank2_update(const uint16_t* dA, const uint16_t* dB, const int* ex, int m, int kb,
                           zd* A, int n, int o, int ct0, int nct, int* err, cudaStream_t s) {
  // 128 x 32 tiles (16 complex columns), four A stages: 97 KB of shared
  // memory and 256 TMEM columns per CTA, two CTAs per SM (16-wide tiles at
  // three CTAs per SM measured 11 % slower: each A tile then serves half the
  // columns)
  constexpr int BN = 32, R2_STAGES = 4, MINB = 2, NT = 256;
  if (((uintptr_t)dA & 15) || ((uintptr_t)dB & 15) || m < 1 || kb < 1 || kb > 65535) {
    bs_set_error("rank-2 update: bad operands (m = %d, batch = %d)", m, kb);
    return BS_EINVAL;
  }
  const int K = R2_S * BK;
  CUtensorMap ta, tb;
  int r = make_map(&ta, dA, K, m, kb, (long)m * K, BM);
  if (!r) r = make_map(&tb, dB, K, 2 * m, kb, (long)2 * m * K, BN);
  if (r) return r;
  const int smem = R2_STAGES * TILE_A + R2_S * tile_b(BN) + 1024;
  static_assert(BM * (BN / 2 + 1) * (int)sizeof(zd) <= R2_STAGES * TILE_A,
                "the staged tile fits in the A ring");
  static std::atomic<bool> attr[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (!attr[dev].load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(rank2_update_kernel<BN, R2_STAGES, MINB, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return bs_cuda_status(e, "rank-2 update smem");
    attr[dev].store(true, std::memory_order_release);
  }
  static_assert(BN == 32, "bs_rank2_column_tiles assumes 32 real columns per tile");
  const int tiles = (2 * m + BN - 1) / BN;
  if (nct <= 0 || ct0 + nct > tiles) nct = tiles - ct0;
  if (nct <= 0) return BS_OK;
  dim3 grid((m + BM - 1) / BM, nct, kb);
  rank2_update_kernel<BN, R2_STAGES, MINB, NT><<<grid, NT, smem, s>>>(ta, tb, ex, m, A, n, o,
                                                                       ct0, err);
  BS_CHECK_LAUNCH("rank2_update_kernel");
  return BS_OK;
}
