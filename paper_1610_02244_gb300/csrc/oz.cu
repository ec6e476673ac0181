// FP64-accurate complex GEMM on the TF32 tensor cores by exact integer slicing.
//
// GB300 runs FP64 FMA at 1.25 TFLOP/s, and its tensor cores run TF32 about 750 times faster. The
// large FP64 products of the update (the FP64 H_eff.theta of the accuracy win-back, theta,
// the environments and the SVD projections) are therefore computed as sums of exact
// integer products (the Ozaki splitting):
//   * every row i of A gets a power-of-two scale sigma_i >= max_k |A_ik| (re and im), every
//     column j of B a scale tau_j, so that A_ik / sigma_i lies in (-1, 1);
//   * A_ik / sigma_i = sum_{p=1..S} a_p 2^{-p beta} + r with integers |a_p| < 2^beta taken by
//     repeated truncation (exact FP64 steps) and |r| < 2^{-S beta}; likewise B;
//   * the slice products a_p b_q are integers below 2^{2 beta}; a K-chunk of them summed
//     over all pairs (p, q) of one level p + q = l stays below 2^24, so TF32 operands
//     (11 significant bits hold |a| < 2^6 exactly) with FP32 accumulation give the level's
//     sum exactly;
//   * C = sum over chunks and levels l = 2..S+1 of 2^{-l beta} sigma_i tau_j (level sum),
//     added in FP64.
// With beta = 6 and S = 9 the pairs kept (p + q <= S + 1) carry 54 bits; the omitted
// terms and the remainders are below (S + 2) 2^{-54} K sigma_i tau_j, the size of an FP64
// GEMM's own rounding bound.  Complex products take four real MMAs per k step
// (re+ += Ar Br, re- += Ai Bi, im += Ar Bi + Ai Br; re = re+ - re- in FP64).
//
// Kernel: persistent, one CTA per SM over (output tile, level group, K split) items,
// 128 x 128 or 128 x 64 tiles (K is split only when the tiles alone would leave most SMs
// idle, as for the 256 x 256 products of a truncated SVD); warp 0 issues TMA loads of the
// slice planes (3-D maps [plane][row][k], 64-byte swizzle), warp 1 the MMAs into three
// TMEM accumulators, warps 2..5 convert each (chunk, level) accumulator and add it to the
// item's FP64 partial tile, handing TMEM back through an mbarrier; a second kernel adds the
// partial outputs in a fixed order.  All waits bounded.
#include <algorithm>
#include <cmath>
#include <vector>

#include "heff_plan.cuh"
#include "tc_common.cuh"
#include "f32conv.cuh"

namespace tnt {

namespace {
using namespace tc;

constexpr int OZ_S = 9;         // slices per operand
constexpr int OZ_BETA = 6;      // bits per slice
constexpr int OZ_KC = 224;      // K chunk: 2 * S * KC * (2^beta - 1)^2 < 2^24
constexpr int OZ_PLANES = 2 * OZ_S;
constexpr int O_TILE_A = 128 * 16 * 4;               // one A plane tile, 8 KB
// the levels of a tile in two groups of nearly equal work (21 and 24 slice pairs), each
// group an independent work item with its own FP64 partial output
constexpr int OZ_GROUP_SPLIT = 7;                    // levels 2..7 | 8..S+1

template <int BN>
struct OzCfg {
  static constexpr int TILE_B = BN * 16 * 4;
  static constexpr int STAGE = 2 * O_TILE_A + 2 * TILE_B;  // A re, A im, B re, B im
  static constexpr int STAGES = (BN == 128) ? 6 : 8;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
  static constexpr int TMEM = (BN == 128) ? 512 : 256;
};
static_assert(2LL * OZ_S * OZ_KC * ((1 << OZ_BETA) - 1) * ((1 << OZ_BETA) - 1) < (1LL << 24),
              "a level sum over one K chunk must stay exact in FP32");
static_assert(OZ_KC % 16 == 0, "K chunk in whole k-blocks");

struct OzArgs {
  int64_t M, N, Kp;
  int ntm, ntn;       // tiles along M and N
  int nchunk;         // K chunks of OZ_KC
  int ks;             // K splits: split s takes chunks [s nchunk / ks, (s+1) nchunk / ks)
  z* P;               // 2 ks FP64 partial outputs, [split][group][M][N]
  const double* sA;   // row scales (powers of two)
  const double* sB;   // column scales
  int* status;
};

// sub-items of one tile: (chunk, level), levels 2..S+1; pairs (p, l - p), 1 <= p, q <= S
__device__ __forceinline__ void level_pairs(int l, int* p0, int* p1) {
  *p0 = max(1, l - OZ_S);
  *p1 = min(OZ_S, l - 1);
}

template <int BN>
__global__ void __launch_bounds__(192, 1) k_oz_gemm(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB,
                                                    OzArgs g) {
  using Cf = OzCfg<BN>;
  constexpr int O_STAGES = Cf::STAGES;
  constexpr int O_STAGE = Cf::STAGE;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + O_STAGES * O_STAGE);
  uint64_t* empty = full + O_STAGES;
  uint64_t* accf = empty + O_STAGES;
  uint64_t* acce = accf + 1;
  uint32_t* tmem_slot = (uint32_t*)(acce + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = g.ntm * g.ntn;
  const int nitems = 2 * ntiles * g.ks;  // (tile, level group, K split)
  const int kb_total = (int)(g.Kp / 16);
  const int kb_chunk = OZ_KC / 16;

  if (threadIdx.x == 0) {
    for (int s = 0; s < O_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 4);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(Cf::TMEM)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer
    uint32_t it = 0;
    bool stop = false;
    for (int w = blockIdx.x; w < nitems && !stop; w += gridDim.x) {
      const int t = w % ntiles, grp = (w / ntiles) & 1, sp = w / (2 * ntiles);
      const int m0 = (t / g.ntn) * 128, n0 = (t % g.ntn) * BN;
      const int l0 = grp ? OZ_GROUP_SPLIT + 1 : 2, l1 = grp ? OZ_S + 1 : OZ_GROUP_SPLIT;
      const int ch0 = sp * g.nchunk / g.ks, ch1 = (sp + 1) * g.nchunk / g.ks;
      for (int ch = ch0; ch < ch1 && !stop; ++ch) {
        const int kb0 = ch * kb_chunk, kb1 = min(kb_total, kb0 + kb_chunk);
        for (int l = l0; l <= l1 && !stop; ++l) {
          int p0, p1;
          level_pairs(l, &p0, &p1);
          for (int p = p0; p <= p1 && !stop; ++p) {
            const int q = l - p;
            for (int kb = kb0; kb < kb1; ++kb) {
              const int s = it % O_STAGES;
              if (it >= O_STAGES && !mbar_wait(&empty[s], ((it / O_STAGES) & 1) ^ 1, g.status)) {
                *abort_flag = 1;
                stop = true;
                break;
              }
              if (*abort_flag) {
                stop = true;
                break;
              }
              uint8_t* st = smem + s * O_STAGE;
              mbar_expect_tx(&full[s], O_STAGE);
              const int k = kb * 16;
              tma_load3(st, &tmA, &full[s], k, m0, 2 * (p - 1));
              tma_load3(st + O_TILE_A, &tmA, &full[s], k, m0, 2 * (p - 1) + 1);
              tma_load3(st + 2 * O_TILE_A, &tmB, &full[s], k, n0, 2 * (q - 1));
              tma_load3(st + 2 * O_TILE_A + Cf::TILE_B, &tmB, &full[s], k, n0, 2 * (q - 1) + 1);
              ++it;
            }
          }
        }
      }
    }
    for (uint32_t i = (it > (uint32_t)O_STAGES ? it - O_STAGES : 0u); i < it; ++i)
      mbar_wait(&full[i % O_STAGES], (i / O_STAGES) & 1, g.status);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issuer
    const uint32_t id = idesc_tf32_n(BN);
    const uint32_t t_re = tmem, t_im = tmem + BN, t_rn = tmem + 2 * BN;
    uint32_t it = 0, sub = 0;
    bool stop = false;
    for (int w = blockIdx.x; w < nitems && !stop; w += gridDim.x) {
      const int grp = (w / ntiles) & 1, sp = w / (2 * ntiles);
      const int l0 = grp ? OZ_GROUP_SPLIT + 1 : 2, l1 = grp ? OZ_S + 1 : OZ_GROUP_SPLIT;
      const int ch0 = sp * g.nchunk / g.ks, ch1 = (sp + 1) * g.nchunk / g.ks;
      for (int ch = ch0; ch < ch1 && !stop; ++ch) {
        const int kb0 = ch * kb_chunk, kb1 = min(kb_total, kb0 + kb_chunk);
        for (int l = l0; l <= l1 && !stop; ++l) {
          int p0, p1;
          level_pairs(l, &p0, &p1);
          if (sub > 0 && (*abort_flag || !mbar_wait(acce, (sub - 1) & 1, g.status))) {
            *abort_flag = 1;
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          bool first = true;
          for (int p = p0; p <= p1 && !stop; ++p) {
            for (int kb = kb0; kb < kb1; ++kb) {
              const int s = it % O_STAGES;
              if (*abort_flag || !mbar_wait(&full[s], (it / O_STAGES) & 1, g.status)) {
                *abort_flag = 1;
                stop = true;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              const uint32_t base = su32(smem + s * O_STAGE);
              for (int ks = 0; ks < 2; ++ks) {
                const uint32_t off = ks * 32;
                const uint64_t ar = desc_sw64(base + off);
                const uint64_t ai = desc_sw64(base + O_TILE_A + off);
                const uint64_t br = desc_sw64(base + 2 * O_TILE_A + off);
                const uint64_t bi = desc_sw64(base + 2 * O_TILE_A + Cf::TILE_B + off);
                const uint32_t acc = first ? 0u : 1u;
                mma_tf32(t_re, ar, br, id, acc);
                mma_tf32(t_rn, ai, bi, id, acc);
                mma_tf32(t_im, ar, bi, id, acc);
                mma_tf32(t_im, ai, br, id, 1);
                first = false;
              }
              mma_commit(&empty[s]);
              ++it;
            }
          }
          if (stop) break;
          mma_commit(accf);
          ++sub;
        }
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue: level sums into FP64 C
    const int q4 = warp & 3;
    const int row = q4 * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(q4 * 32) << 16;
    uint32_t sub = 0;
    bool stop = false;
    for (int w = blockIdx.x; w < nitems && !stop; w += gridDim.x) {
      const int t = w % ntiles, grp = (w / ntiles) & 1, sp = w / (2 * ntiles);
      const int m0 = (t / g.ntn) * 128, n0 = (t % g.ntn) * BN;
      const int l0 = grp ? OZ_GROUP_SPLIT + 1 : 2, l1 = grp ? OZ_S + 1 : OZ_GROUP_SPLIT;
      const int64_t gm = (int64_t)m0 + row;
      const double sa = (gm < g.M) ? g.sA[gm] : 0.0;
      z* Cg = g.P + (int64_t)(grp + 2 * sp) * g.M * g.N;
      const int ch0 = sp * g.nchunk / g.ks, ch1 = (sp + 1) * g.nchunk / g.ks;
      for (int ch = ch0; ch < ch1 && !stop; ++ch) {
        for (int l = l0; l <= l1; ++l) {
          if (*abort_flag || !mbar_wait(accf, sub & 1, g.status)) {
            *abort_flag = 1;
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const double lv = ldexp(sa, -l * OZ_BETA);
          const bool first = (ch == ch0 && l == l0);
          for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t r[32], s[32], u[32];
            tmem_ld32(tmem + lane_addr + c0, r);
            tmem_ld32(tmem + lane_addr + BN + c0, s);
            tmem_ld32(tmem + lane_addr + 2 * BN + c0, u);
            if (gm < g.M) {
              z* pc = Cg + gm * g.N + n0 + c0;
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const int64_t gn = (int64_t)n0 + c0 + j;
                if (gn < g.N) {
                  const double f = lv * g.sB[gn];
                  const double dr = (double)__uint_as_float(r[j]) - (double)__uint_as_float(u[j]);
                  const double di = (double)__uint_as_float(s[j]);
                  if (first) {
                    pc[j] = zmk(dr * f, di * f);
                  } else {
                    const z o = pc[j];
                    pc[j] = zmk(fma(dr, f, o.x), fma(di, f, o.y));
                  }
                }
              }
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(acce);
          ++sub;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cf::TMEM)
                 : "memory");
  }
}

// C = P[0] + P[1], the two level groups, in a fixed order
__global__ void k_oz_finish(const z* __restrict__ P, int np, int64_t M, int64_t N,
                            z* __restrict__ C, int64_t ldc) {
  const int64_t total = M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    z acc = P[e];
    for (int i = 1; i < np; ++i) acc = zadd(acc, P[(int64_t)i * total + e]);
    C[(e / N) * ldc + e % N] = acc;
  }
}

// ---------------------------------------------------------------- scales and slices
// sA[i] = 2^e with 2^(e-1) <= max_k max(|re A_ik|, |im A_ik|) < 2^e (1 for a zero row);
// one warp per row of a strided operand X[i * rs + k * cs]
__global__ void k_oz_row_scale(const z* __restrict__ X, int64_t rows, int64_t K, int64_t rs,
                               int64_t cs, double* __restrict__ sc) {
  // by integer operations on the exponent fields (no FP64-pipe comparisons): the largest
  // field mx of the row gives 2^(mx - 1023) <= max < 2^(mx - 1022), so sc = 2^(mx - 1022),
  // the frexp exponent of the maximum; a row of subnormals gets 2^-1022, a zero row 1
  const int lane = threadIdx.x & 31;
  for (int64_t i = (int64_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); i < rows;
       i += (int64_t)((gridDim.x * blockDim.x) >> 5)) {
    unsigned mx = 0, nz = 0;
    for (int64_t k = lane; k < K; k += 32) {
      const z v = X[i * rs + k * cs];
      const unsigned hr = (unsigned)__double2hiint(v.x), hi = (unsigned)__double2hiint(v.y);
      mx = max(mx, max((hr >> 20) & 0x7ffu, (hi >> 20) & 0x7ffu));
      nz |= (hr & 0x7fffffffu) | (unsigned)__double2loint(v.x) | (hi & 0x7fffffffu) |
            (unsigned)__double2loint(v.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      nz |= __shfl_xor_sync(0xffffffffu, nz, o);
    }
    if (lane == 0) {
      double r = 1.0;
      if (mx > 0) r = __hiloint2double((int)((mx + 1u) << 20), 0);  // 2^(mx - 1022)
      else if (nz) r = __hiloint2double(1 << 20, 0);                  // 2^-1022
      sc[i] = r;
    }
  }
}

// slice planes: out[2(p-1) + (0 re | 1 im)][i][k] = p-th integer slice of X_ik / sc[i],
// i < rows, k < Kp (zero for k >= K); X[i * rs + k * cs], conjugated if conj
static_assert(OZ_S * OZ_BETA == 54, "the fixed-point form holds 54 bits");
__global__ void k_oz_slice(const z* __restrict__ X, int64_t rows, int64_t K, int64_t Kp,
                           int64_t rs, int64_t cs, int conj, const double* __restrict__ sc,
                           float* __restrict__ out) {
  // The p-th slice is the p-th base-2^beta digit of X_ik / sc[i] with its sign: what
  // repeated multiplication by 2^beta and truncation give (every step exact), taken here
  // from the fixed-point value F = floor(|X_ik| / sc[i] 2^54) by shifts and masks
  const int64_t plane = rows * Kp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < plane;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / Kp, k = e % Kp;
    uint64_t fr = 0, fi = 0;
    bool nr = false, ni = false;
    if (k < K) {
      const z v = X[i * rs + k * cs];
      const int esc = (int)(((uint64_t)__double_as_longlong(sc[i]) >> 52) & 0x7ff) - 1023;
      fr = fixed54(v.x, esc);
      fi = fixed54(v.y, esc);
      nr = __double2hiint(v.x) < 0;
      ni = (__double2hiint(v.y) < 0) != (conj != 0);
    }
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) {
      const int shift = OZ_S * OZ_BETA - OZ_BETA * (p + 1);
      const float ar = (float)(int)((fr >> shift) & ((1u << OZ_BETA) - 1));
      const float ai = (float)(int)((fi >> shift) & ((1u << OZ_BETA) - 1));
      out[(int64_t)(2 * p) * plane + e] = nr ? -ar : ar;
      out[(int64_t)(2 * p + 1) * plane + e] = ni ? -ai : ai;
    }
  }
}

unsigned ogrid(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }
int64_t rup16(int64_t x) { return (x + 15) / 16 * 16; }

}  // namespace

size_t ozgemm_scratch_bytes(int64_t M, int64_t N, int64_t K, int ks) {
  const int64_t Kp = rup16(K);
  return ws_round(sizeof(float) * OZ_PLANES * M * Kp) + ws_round(sizeof(float) * OZ_PLANES * N * Kp) +
         ws_round(sizeof(double) * M) + ws_round(sizeof(double) * N) +
         ws_round(sizeof(z) * 2 * (size_t)ks * M * N) + 4096;
}

bool ozgemm_eligible(const Ctx* c, const ZGemm& g) {
  // (a Hermitian product asked for its lower part only is formed whole: the caller mirrors it)
  return c->oz_mode != 0 && g.batch == 1 && g.alpha.x == 1.0 && g.alpha.y == 0.0 &&
         g.beta.x == 0.0 && g.beta.y == 0.0 && g.M >= 128 && g.N >= 64 && g.K >= 64 &&
         (double)g.M * (double)g.N * (double)g.K >= 3.0e7 && g.M < (1LL << 31) && g.N < (1LL << 31);
}

namespace {
template <int BN>
int launch_oz(Ctx* c, const CUtensorMap& tA, const CUtensorMap& tB, const OzArgs& a, int nitems, int sm) {
  static bool attr = false;
  if (!attr) {
    TNT_CUDA_TRY(c, cudaFuncSetAttribute(k_oz_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         OzCfg<BN>::SMEM));
    attr = true;
  }
  k_oz_gemm<BN><<<(unsigned)std::min(nitems, sm), 192, OzCfg<BN>::SMEM, c->stream>>>(tA, tB, a);
  return TNT_OK;
}
}  // namespace

// C = A B (FP64-accurate) through the integer-slice tensor-core kernel; slices and the two
// partial outputs live in the context's own buffer (grown between calls, never inside a
// capture)
int ozgemm(Ctx* c, const ZGemm& g) {
  const int64_t M = g.M, N = g.N, K = g.K, Kp = rup16(K);
  static int sm = 0;
  if (!sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sm < 1) sm = 152;
  }
  const int ntm = (int)((M + 127) / 128);
  // N tile 64 when 128-wide tiles would leave SMs idle; split K when even the 64-wide
  // (tile, level group) items leave most SMs idle (a 256 x 256 product makes 16), keeping
  // the partial outputs within 256 MB
  const int bn = (2LL * ntm * ((N + 127) / 128) < 2LL * sm) ? 64 : 128;
  const int ntn = (int)((N + bn - 1) / bn);
  const int nchunk = (int)((Kp + OZ_KC - 1) / OZ_KC);
  int ks = 1;
  if (2LL * ntm * ntn < sm) ks = (int)std::min<int64_t>(nchunk, std::max<int64_t>(1, sm / (2LL * ntm * ntn)));
  while (ks > 1 && 32.0 * ks * (double)M * (double)N > 256e6) --ks;
  const size_t need = ozgemm_scratch_bytes(M, N, K, ks);
  if (need > c->oz_cap) {
    TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    dev_free(c->dalloc, c->oz_buf);
    c->oz_buf = nullptr;
    c->oz_cap = 0;
    if (dev_alloc(c->dalloc, &c->oz_buf, need) != 0)
      return set_err(c, TNT_E_ALLOC, "device allocation of %zu bytes (FP64 product slices) failed", need);
    c->oz_cap = need;
  }
  char* b = (char*)c->oz_buf;
  float* Ap = (float*)b;
  b += ws_round(sizeof(float) * OZ_PLANES * M * Kp);
  float* Bp = (float*)b;
  b += ws_round(sizeof(float) * OZ_PLANES * N * Kp);
  double* sA = (double*)b;
  b += ws_round(sizeof(double) * M);
  double* sB = (double*)b;
  b += ws_round(sizeof(double) * N);
  z* P = (z*)b;
  // B enters as rows n with K along the row: B^T[n][k] = B[k * b_rs + n * b_cs]
  k_oz_row_scale<<<ogrid(32 * M), 256, 0, c->stream>>>(g.A, M, K, g.a_rs, g.a_cs, sA);
  k_oz_row_scale<<<ogrid(32 * N), 256, 0, c->stream>>>(g.B, N, K, g.b_cs, g.b_rs, sB);
  {
    ProfScope ps(c, "oz_slice", 16.0 * (double)(M + N) * (double)K + 4.0 * OZ_PLANES * (double)(M + N) * Kp);
    k_oz_slice<<<ogrid(M * Kp), 256, 0, c->stream>>>(g.A, M, K, Kp, g.a_rs, g.a_cs, g.conj_a, sA, Ap);
    k_oz_slice<<<ogrid(N * Kp), 256, 0, c->stream>>>(g.B, N, K, Kp, g.b_cs, g.b_rs, g.conj_b, sB, Bp);
  }
  c->launches += 4;
  TNT_CHECK_LAUNCH(c);
  OzArgs a;
  a.M = M;
  a.N = N;
  a.Kp = Kp;
  a.nchunk = nchunk;
  a.ks = ks;
  a.ntm = ntm;
  a.ntn = ntn;
  a.P = P;
  a.sA = sA;
  a.sB = sB;
  a.status = c->d_status;
  CUtensorMap tA, tB;
  TNT_TRY(tma_map_planes_n(c, &tA, Ap, M, Kp, 128, OZ_PLANES));
  TNT_TRY(tma_map_planes_n(c, &tB, Bp, N, Kp, bn, OZ_PLANES));
  const int nitems = 2 * a.ntm * a.ntn * ks;
  {
    ProfScope ps(c, "oz_gemm", 8.0 * (double)M * (double)N * (double)K);
    TNT_TRY(bn == 64 ? launch_oz<64>(c, tA, tB, a, nitems, sm) : launch_oz<128>(c, tA, tB, a, nitems, sm));
    k_oz_finish<<<ogrid(M * N), 256, 0, c->stream>>>(P, 2 * ks, M, N, g.C, g.c_rs);
  }
  c->launches += 2;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

}  // namespace tnt
