// Grouped launches of the U(1) block-sparse H_eff.theta (block structure: App. A.1.1 and
// App. B.1.2; contraction order: Sec. 4.2 Listing 1 in two-site form).
//
// One matvec over every block of every problem is five launches (split TF32) or four
// (FP64), whatever the number of charge sectors or problems:
//   pack   theta slabs -> transposed split-TF32 planes (mixed only)
//   GEMM 1 T1 = L . theta, all (problem, left sector) tasks in one persistent launch
//   W      T3 = W1 W2 . T1 over all (a' sector, b sector) pairs
//   GEMM 4 Y = T3 . R^T, all (problem, right sector) tasks in one persistent launch
//   gather Y rows -> compact y (sum of the split-K parts in a fixed order)
// The persistent tcgen05 kernel walks a tile list (task, m0, n0, split); one CTA per SM,
// TMA producer warp, MMA warp, four epilogue warps, 3-4 stage smem ring, one TMEM
// accumulator set that the epilogue hands back through an mbarrier.  Tile N (64 or 128)
// and the split-K of GEMM 4 are chosen by timing the candidates once per block-structure
// signature.  The launches are recorded once as a CUDA graph; a replay patches the input
// and output pointers of the first and last node.
#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "heff_plan.cuh"
#include "tc_common.cuh"
#include "u1.cuh"

namespace tnt {

namespace {
using namespace tc;

template <int BN>
struct GCfg {
  static constexpr int TILE_A = 128 * 16 * 4;
  static constexpr int TILE_B = BN * 16 * 4;
  static constexpr int STAGE = 4 * TILE_A + 4 * TILE_B;
  static constexpr int STAGES = (BN == 128) ? 3 : 4;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
  static constexpr int TMEM_COLS = (BN == 128) ? 512 : 256;
};

// ---------------------------------------------------------------- grouped tcgen05 GEMM
template <int BN>
__global__ void __launch_bounds__(192, 1) k_cgemm_grouped(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB,
                                                          GArgs g) {
  using Cf = GCfg<BN>;
  constexpr int STAGES = Cf::STAGES;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * Cf::STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;  // accumulators complete
  uint64_t* acce = accf + 1;        // accumulators read out by the epilogue
  uint32_t* tmem_slot = (uint32_t*)(acce + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
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
                 "r"(Cf::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer over all my tiles
    uint32_t it = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < g.ntiles && !stop; t += gridDim.x) {
      const int4 tl = g.tiles[t];
      const GTask tk = g.tasks[tl.x];
      const int kb0 = tl.w * tk.kb_per_split;
      const int kb1 = min(tk.kb_total, kb0 + tk.kb_per_split);
      for (int kb = kb0; kb < kb1; ++kb) {
        const int s = it % STAGES;
        if (it >= STAGES && !mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1, g.status)) {
          *abort_flag = 1;
          stop = true;
          break;
        }
        if (*abort_flag) {
          stop = true;
          break;
        }
        uint8_t* st = smem + s * Cf::STAGE;
        mbar_expect_tx(&full[s], Cf::STAGE);
        const int k = kb * 16;
        for (int p = 0; p < 4; ++p)
          tma_load3(st + p * Cf::TILE_A, &tmA, &full[s], k, tk.a_row0 + tl.y, p);
        for (int p = 0; p < 4; ++p)
          tma_load3(st + 4 * Cf::TILE_A + p * Cf::TILE_B, &tmB, &full[s], k, tk.b_row0 + tl.z, p);
        ++it;
      }
    }
    // every stage filled must have landed before the CTA may exit
    for (uint32_t i = (it > (uint32_t)STAGES ? it - STAGES : 0u); i < it; ++i)
      mbar_wait(&full[i % STAGES], (i / STAGES) & 1, g.status);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issuer
    const uint32_t id = idesc_tf32_n(BN);
    const uint32_t t_re = tmem, t_im = tmem + BN, t_rn = tmem + 2 * BN;
    uint32_t it = 0, tc = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < g.ntiles && !stop; t += gridDim.x) {
      const int4 tl = g.tiles[t];
      const GTask tk = g.tasks[tl.x];
      const int kb0 = tl.w * tk.kb_per_split;
      const int kb1 = min(tk.kb_total, kb0 + tk.kb_per_split);
      if (tc > 0 && (*abort_flag || !mbar_wait(acce, (tc - 1) & 1, g.status))) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int kb = kb0; kb < kb1; ++kb) {
        const int s = it % STAGES;
        if (*abort_flag || !mbar_wait(&full[s], (it / STAGES) & 1, g.status)) {
          *abort_flag = 1;
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = su32(smem + s * Cf::STAGE);
        for (int ks = 0; ks < 2; ++ks) {  // K = 8 per tf32 MMA: 32 bytes along the row
          const uint32_t off = ks * 32;
          const uint64_t a_rh = desc_sw64(base + 0 * Cf::TILE_A + off);
          const uint64_t a_rl = desc_sw64(base + 1 * Cf::TILE_A + off);
          const uint64_t a_ih = desc_sw64(base + 2 * Cf::TILE_A + off);
          const uint64_t a_il = desc_sw64(base + 3 * Cf::TILE_A + off);
          const uint32_t bb = base + 4 * Cf::TILE_A;
          const uint64_t b_rh = desc_sw64(bb + 0 * Cf::TILE_B + off);
          const uint64_t b_rl = desc_sw64(bb + 1 * Cf::TILE_B + off);
          const uint64_t b_ih = desc_sw64(bb + 2 * Cf::TILE_B + off);
          const uint64_t b_il = desc_sw64(bb + 3 * Cf::TILE_B + off);
          const uint32_t first = (kb == kb0 && ks == 0) ? 0u : 1u;
          mma_tf32(t_re, a_rh, b_rh, id, first);
          mma_tf32(t_re, a_rh, b_rl, id, 1);
          mma_tf32(t_re, a_rl, b_rh, id, 1);
          mma_tf32(t_rn, a_ih, b_ih, id, first);
          mma_tf32(t_rn, a_ih, b_il, id, 1);
          mma_tf32(t_rn, a_il, b_ih, id, 1);
          mma_tf32(t_im, a_rh, b_ih, id, first);
          mma_tf32(t_im, a_rh, b_il, id, 1);
          mma_tf32(t_im, a_rl, b_ih, id, 1);
          mma_tf32(t_im, a_ih, b_rh, id, 1);
          mma_tf32(t_im, a_ih, b_rl, id, 1);
          mma_tf32(t_im, a_il, b_rh, id, 1);
        }
        mma_commit(&empty[s]);
        ++it;
      }
      if (stop) break;
      mma_commit(accf);
      ++tc;
    }
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue: TMEM -> global (FP32)
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
    uint32_t tc = 0;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
      if (*abort_flag || !mbar_wait(accf, tc & 1, g.status)) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int4 tl = g.tiles[t];
      const GTask tk = g.tasks[tl.x];
      const int64_t gm = (int64_t)tl.y + row;
      float* Cre = g.C + tk.c_off + (int64_t)tl.w * g.split_stride;
      float* Cim = Cre + g.plane;
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32], s[32], u[32];
        tmem_ld32(tmem + lane_addr + c0, r);
        tmem_ld32(tmem + lane_addr + BN + c0, s);
        tmem_ld32(tmem + lane_addr + 2 * BN + c0, u);
        if (gm < tk.M) {
          float* pr = Cre + gm * tk.ldc + tl.z + c0;
          float* pi = Cim + gm * tk.ldc + tl.z + c0;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (tl.z + c0 + j < tk.N) {
              pr[j] = __uint_as_float(r[j]) - __uint_as_float(u[j]);
              pi[j] = __uint_as_float(s[j]);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(acce);
      ++tc;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(Cf::TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- grouped FP64 GEMM
constexpr int ZM = 64, ZN = 64, ZK = 16;
__global__ void __launch_bounds__(256) k_zgemm_grouped(ZGArgs g) {
  __shared__ z As[ZK][ZM + 1];
  __shared__ z Bs[ZK][ZN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    const int4 tl = g.tiles[t];
    const ZTask tk = g.tasks[tl.x];
    const int64_t m0 = tl.y, n0 = tl.z;
    const z* A = g.A + tk.a_off;
    const z* B = g.B + tk.b_off;
    z acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] = zmk(0, 0);
    const bool a_kfast = (tk.a_cs == 1), b_nfast = (tk.b_cs == 1);
    for (int64_t k0 = 0; k0 < tk.K; k0 += ZK) {
#pragma unroll
      for (int u = 0; u < (ZM * ZK) / 256; ++u) {
        const int e = threadIdx.x + 256 * u;
        int i, k;
        if (a_kfast) { k = e % ZK; i = e / ZK; } else { i = e % ZM; k = e / ZM; }
        const int64_t gi = m0 + i, gk = k0 + k;
        As[k][i] = (gi < tk.M && gk < tk.K) ? A[gi * tk.a_rs + gk * tk.a_cs] : zmk(0, 0);
      }
#pragma unroll
      for (int u = 0; u < (ZN * ZK) / 256; ++u) {
        const int e = threadIdx.x + 256 * u;
        int j, k;
        if (b_nfast) { j = e % ZN; k = e / ZN; } else { k = e % ZK; j = e / ZK; }
        const int64_t gj = n0 + j, gk = k0 + k;
        Bs[k][j] = (gj < tk.N && gk < tk.K) ? B[gk * tk.b_rs + gj * tk.b_cs] : zmk(0, 0);
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < ZK; ++kk) {
        z a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
        for (int q = 0; q < 4; ++q) b[q] = Bs[kk][tx + 16 * q];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) zfma(acc[r][q], a[r], b[q]);
      }
      __syncthreads();
    }
    z* C = g.C + tk.c_off;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t gi = m0 + ty + 16 * r;
      if (gi >= tk.M) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t gj = n0 + tx + 16 * q;
        if (gj < tk.N) C[gi * tk.c_rs + gj] = acc[r][q];
      }
    }
  }
}

// the same over 16 x 16 tiles, one output per thread: for block structures whose 64 x 64
// tiles would leave most SMs without FP64 work
__global__ void __launch_bounds__(256) k_zgemm_grouped16(ZGArgs g) {
  __shared__ z As[16][17];
  __shared__ z Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    const int4 tl = g.tiles[t];
    const ZTask tk = g.tasks[tl.x];
    const z* A = g.A + tk.a_off;
    const z* B = g.B + tk.b_off;
    z acc = zmk(0, 0);
    for (int64_t k0 = 0; k0 < tk.K; k0 += 16) {
      {
        const int64_t gi = tl.y + ty, gk = k0 + tx;
        As[ty][tx] = (gi < tk.M && gk < tk.K) ? A[gi * tk.a_rs + gk * tk.a_cs] : zmk(0, 0);
      }
      {
        const int64_t gk = k0 + ty, gj = tl.z + tx;
        Bs[ty][tx] = (gj < tk.N && gk < tk.K) ? B[gk * tk.b_rs + gj * tk.b_cs] : zmk(0, 0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) zfma(acc, As[ty][kk], Bs[kk][tx]);
      __syncthreads();
    }
    const int64_t gi = tl.y + ty, gj = tl.z + tx;
    if (gi < tk.M && gj < tk.N) g.C[tk.c_off + gi * tk.c_rs + gj] = acc;
  }
}

// ---------------------------------------------------------------- operand packing
// constant operands (environments): one warp per segment
template <bool MIXED>
__global__ void k_pack_segs(const PackSeg* segs, int nseg, float* dst4, int64_t plane, z* dstz) {
  const int lane = threadIdx.x & 31;
  for (int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); s < nseg;
       s += (int)((gridDim.x * blockDim.x) >> 5)) {
    const PackSeg sg = segs[s];
    for (int64_t i = lane; i < sg.len; i += 32) {
      const z v = sg.src[i];
      if (MIXED) {
        float a, b, c, d;
        split_tf32(v.x, &a, &b);
        split_tf32(v.y, &c, &d);
        float* o = dst4 + sg.dst + i;
        o[0] = a;
        o[plane] = b;
        o[2 * plane] = c;
        o[3 * plane] = d;
      } else {
        dstz[sg.dst + i] = v;
      }
    }
  }
}

// theta slabs [K][N] -> planes[p][dst_row0 + n][k]: 32 x 32 tiles through shared memory
__global__ void __launch_bounds__(256) k_pack_theta_t(TPArgs a) {
  __shared__ z tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int4 tl = a.tiles[t];
    const TSlab sb = a.slabs[tl.x];
    const int64_t n0 = tl.y, k0 = tl.z;
    for (int j = ty; j < 32; j += 8) {
      const int64_t k = k0 + j, n = n0 + tx;
      tile[j][tx] = (k < sb.K && n < sb.N) ? a.x[sb.src + k * sb.N + n] : zmk(0, 0);
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
      const int64_t n = n0 + j, k = k0 + tx;
      if (n < sb.N && k < sb.K) {
        const z v = tile[tx][j];
        float p0, p1, p2, p3;
        split_tf32(v.x, &p0, &p1);
        split_tf32(v.y, &p2, &p3);
        float* o = a.dst + (sb.dst_row0 + n) * a.KA + k;
        o[0] = p0;
        o[a.plane] = p1;
        o[2 * a.plane] = p2;
        o[3 * a.plane] = p3;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- W contraction
constexpr int W_MAX_OUT = 256, W_MAX_IN = 1024, W_TILE = 256;
template <bool MIXED>
__global__ void __launch_bounds__(256) k_wop(WArgs a) {
  __shared__ int64_t s_obase[W_MAX_OUT];
  __shared__ int s_r0[W_MAX_OUT], s_r1[W_MAX_OUT];
  __shared__ int64_t s_ibase[W_MAX_IN];
  __shared__ int64_t s_irs[W_MAX_IN];
  __shared__ z s_val[W_MAX_IN];
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int2 tl = a.tiles[t];
    const WPair pr = a.pairs[tl.x];
    const int r_first = a.outs[pr.out0].r0;
    const int r_last = a.outs[pr.out0 + pr.nout - 1].r1;
    for (int i = threadIdx.x; i < pr.nout; i += blockDim.x) {
      const WOut o = a.outs[pr.out0 + i];
      s_obase[i] = o.base;
      s_r0[i] = o.r0 - r_first;
      s_r1[i] = o.r1 - r_first;
    }
    for (int i = threadIdx.x; i < r_last - r_first; i += blockDim.x) {
      const WIn w = a.ins[r_first + i];
      s_ibase[i] = w.base;
      s_irs[i] = w.rs;
      s_val[i] = w.val;
    }
    __syncthreads();
    const int64_t e = (int64_t)tl.y + threadIdx.x;
    if (e < pr.n_a * pr.n_b) {
      const int64_t ia = e / pr.n_b, jb = e % pr.n_b;
      for (int o = 0; o < pr.nout; ++o) {
        const int64_t dst = s_obase[o] + ia * a.out_rs + jb;
        if (MIXED) {
          float xr = 0.f, xi = 0.f;
          for (int r = s_r0[o]; r < s_r1[o]; ++r) {
            const int64_t src = s_ibase[r] + ia * s_irs[r] + jb;
            const float vr = a.t1f[src], vi = a.t1f[a.p1 + src];
            const float wr = (float)s_val[r].x, wi = (float)s_val[r].y;
            xr = fmaf(wr, vr, fmaf(-wi, vi, xr));
            xi = fmaf(wr, vi, fmaf(wi, vr, xi));
          }
          float h, l;
          split_tf32(xr, &h, &l);
          a.a4f[dst] = h;
          a.a4f[a.p4 + dst] = l;
          split_tf32(xi, &h, &l);
          a.a4f[2 * a.p4 + dst] = h;
          a.a4f[3 * a.p4 + dst] = l;
        } else {
          z acc = zmk(0, 0);
          for (int r = s_r0[o]; r < s_r1[o]; ++r)
            zfma(acc, s_val[r], a.t1z[s_ibase[r] + ia * s_irs[r] + jb]);
          a.a4z[dst] = acc;
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- gather
template <bool MIXED>
__global__ void k_gather_u1(GthArgs a) {
  const int lane = threadIdx.x & 31;
  for (int r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); r < a.nrows;
       r += (int)((gridDim.x * blockDim.x) >> 5)) {
    const GRow g = a.rows[r];
    for (int64_t j = lane; j < g.n; j += 32) {
      if (MIXED) {
        float re = 0.f, im = 0.f;  // FP32 partials added in FP32, widened once (tc_mixed.cu)
        for (int s = 0; s < a.nsplit; ++s) {
          re += a.yf[s * a.sstride + g.src + j];
          im += a.yf[s * a.sstride + a.plane + g.src + j];
        }
        a.y[g.dst + j] = zmk(f64_of(re), f64_of(im));
      } else {
        a.y[g.dst + j] = a.yz[g.src + j];
      }
    }
  }
}

// dense <-> compact copies (segments with offsets on both sides)
__global__ void k_copy_runs(const int64_t* runs, int nrun, const z* src, z* dst) {
  const int lane = threadIdx.x & 31;
  for (int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); s < nrun;
       s += (int)((gridDim.x * blockDim.x) >> 5)) {
    const int64_t so = runs[3 * s], dof = runs[3 * s + 1], len = runs[3 * s + 2];
    for (int64_t i = lane; i < len; i += 32) dst[dof + i] = src[so + i];
  }
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 152;
  }
  return n;
}
unsigned cap_grid(int64_t work, int64_t cap) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(work, cap));
}
int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// ---------------------------------------------------------------- host layout
struct Layout {
  std::vector<Sector> Ls, Rs;
  std::map<int64_t, int> Li, Ri;
  std::vector<int64_t> N, toff;               // per left sector
  std::vector<std::vector<int64_t>> coff;     // per left sector, per (s1 s2): -1 if absent
  int64_t n = 0;
};

std::vector<Sector> sectors_of(const std::vector<int64_t>& q) {
  std::vector<Sector> s;
  for (int64_t i = 0; i < (int64_t)q.size(); ++i) {
    if (s.empty() || s.back().q != q[(size_t)i]) s.push_back(Sector{q[(size_t)i], i, 0});
    s.back().size++;
  }
  return s;
}

Layout layout_of(const U1Spec& sp) {
  Layout l;
  l.Ls = sectors_of(sp.qa);
  l.Rs = sectors_of(sp.qb);
  for (int i = 0; i < (int)l.Ls.size(); ++i) l.Li[l.Ls[(size_t)i].q] = i;
  for (int i = 0; i < (int)l.Rs.size(); ++i) l.Ri[l.Rs[(size_t)i].q] = i;
  const int64_t d = sp.d;
  for (const Sector& s : l.Ls) {
    std::vector<int64_t> co((size_t)(d * d), -1);
    int64_t N = 0;
    for (int64_t s1 = 0; s1 < d; ++s1)
      for (int64_t s2 = 0; s2 < d; ++s2) {
        auto it = l.Ri.find(s.q + s1 + s2);
        if (it == l.Ri.end()) continue;
        co[(size_t)(s1 * d + s2)] = N;
        N += l.Rs[(size_t)it->second].size;
      }
    l.coff.push_back(co);
    l.N.push_back(N);
    l.toff.push_back(l.n);
    l.n += s.size * N;
  }
  return l;
}

// tiles of one stage for tile N = bn and split-K = split (split clipped per task so that
// no split is empty)
void make_tiles(const std::vector<TaskDesc>& ts, int bn, int split, std::vector<GTask>* gt,
                std::vector<int4>* tiles) {
  gt->clear();
  tiles->clear();
  for (size_t i = 0; i < ts.size(); ++i) {
    const TaskDesc& t = ts[i];
    GTask g{};
    g.a_row0 = (int)t.a_row0;
    g.b_row0 = (int)t.b_row0;
    g.M = (int)t.M;
    g.N = (int)t.N;
    g.kb_total = (int)((t.K + 15) / 16);
    int sp = std::max(1, std::min(split, g.kb_total));
    int per = (g.kb_total + sp - 1) / sp;
    while (sp > 1 && per * (sp - 1) >= g.kb_total) {
      --sp;
      per = (g.kb_total + sp - 1) / sp;
    }
    g.kb_per_split = per;
    g.c_off = t.c_off;
    g.ldc = t.ldc;
    gt->push_back(g);
    for (int s = 0; s < sp; ++s)
      for (int64_t m0 = 0; m0 < t.M; m0 += 128)
        for (int64_t n0 = 0; n0 < t.N; n0 += bn) tiles->push_back(make_int4((int)i, (int)m0, (int)n0, s));
  }
}

void make_ztiles(const std::vector<ZTask>& ts, int tile, std::vector<int4>* tiles) {
  tiles->clear();
  for (size_t i = 0; i < ts.size(); ++i)
    for (int64_t m0 = 0; m0 < ts[i].M; m0 += tile)
      for (int64_t n0 = 0; n0 < ts[i].N; n0 += tile) tiles->push_back(make_int4((int)i, (int)m0, (int)n0, 0));
}

template <typename T>
int upload(Ctx* c, T** dptr, const std::vector<T>& h, size_t cap_elems = 0) {
  const size_t n = std::max(h.size(), cap_elems);
  *dptr = (T*)ws_alloc(c, ws_round(sizeof(T) * std::max<size_t>(n, 1)));
  if (!*dptr) return set_err(c, TNT_E_ALLOC, "scratch exhausted (grouped matvec tables)");
  if (!h.empty())
    TNT_CUDA_TRY(c, cudaMemcpyAsync(*dptr, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, c->stream));
  return TNT_OK;
}

// host tables kept with the plan for the tiles of the grouped FP64 GEMMs
struct ZHost {
  std::vector<ZTask> z1, z4;
};

template <int BN>
int launch_grouped(Ctx* c, const CUtensorMap& tA, const CUtensorMap& tB, const GArgs& g, int ntiles) {
  using Cf = GCfg<BN>;
  static bool attr = false;
  if (!attr) {
    TNT_CUDA_TRY(c, cudaFuncSetAttribute(k_cgemm_grouped<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM));
    attr = true;
  }
  if (ntiles <= 0) return TNT_OK;
  k_cgemm_grouped<BN><<<cap_grid(ntiles, sm_count()), 192, Cf::SMEM, c->stream>>>(tA, tB, g);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

int launch_grouped_bn(Ctx* c, int bn, const CUtensorMap& tA, const CUtensorMap& tB, const GArgs& g, int ntiles) {
  return bn == 64 ? launch_grouped<64>(c, tA, tB, g, ntiles) : launch_grouped<128>(c, tA, tB, g, ntiles);
}

}  // namespace

// ====================================================================== public (internal)
int u1_check(Ctx* c, const U1Spec& s) {
  if (s.chl < 1 || s.chr < 1 || s.d < 1 || s.D < 1 || !s.L || !s.R || !s.W1 || !s.W2)
    return set_err(c, TNT_E_INVALID, "U(1) problem: bad size or null pointer");
  if ((int64_t)s.qa.size() != s.chl || (int64_t)s.qb.size() != s.chr || (int64_t)s.wq.size() != s.D)
    return set_err(c, TNT_E_INVALID, "U(1) problem: label arrays do not match the sizes");
  for (size_t i = 1; i < s.qa.size(); ++i)
    if (s.qa[i] < s.qa[i - 1]) return set_err(c, TNT_E_INVALID, "left labels must be non-decreasing");
  for (size_t i = 1; i < s.qb.size(); ++i)
    if (s.qb[i] < s.qb[i - 1]) return set_err(c, TNT_E_INVALID, "right labels must be non-decreasing");
  return TNT_OK;
}

int64_t u1_compact_size(const U1Spec& s) { return layout_of(s).n; }

int u1_convert(Ctx* c, const U1Spec& s, const z* src, z* dst, int to_compact) {
  const Layout l = layout_of(s);
  const int64_t d = s.d;
  std::vector<int64_t> runs;
  for (size_t iL = 0; iL < l.Ls.size(); ++iL) {
    const Sector& sa = l.Ls[iL];
    for (int64_t a = 0; a < sa.size; ++a)
      for (int64_t s1 = 0; s1 < d; ++s1)
        for (int64_t s2 = 0; s2 < d; ++s2) {
          const int64_t co = l.coff[iL][(size_t)(s1 * d + s2)];
          if (co < 0) continue;
          const Sector& sb = l.Rs[(size_t)l.Ri.at(sa.q + s1 + s2)];
          const int64_t dense = (((sa.start + a) * d + s1) * d + s2) * s.chr + sb.start;
          const int64_t comp = l.toff[iL] + a * l.N[iL] + co;
          runs.push_back(to_compact ? dense : comp);
          runs.push_back(to_compact ? comp : dense);
          runs.push_back(sb.size);
        }
  }
  if (!to_compact) TNT_TRY(zfill(c, dst, s.chl * d * d * s.chr, zmk(0, 0)));
  const int nrun = (int)(runs.size() / 3);
  if (nrun == 0) return TNT_OK;
  int64_t* d_runs = (int64_t*)ws_alloc(c, ws_round(sizeof(int64_t) * runs.size()));
  if (!d_runs) return set_err(c, TNT_E_ALLOC, "scratch exhausted (block runs)");
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_runs, runs.data(), sizeof(int64_t) * runs.size(), cudaMemcpyHostToDevice, c->stream));
  k_copy_runs<<<cap_grid((nrun + 7) / 8, 152 * 8), 256, 0, c->stream>>>(d_runs, nrun, src, dst);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  // the host run table must outlive the asynchronous copy
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return TNT_OK;
}

U1Plan::~U1Plan() {
  for (int i = 0; i < 2; ++i) {
    if (exec[i]) cudaGraphExecDestroy(exec[i]);
    if (graph[i]) cudaGraphDestroy(graph[i]);
  }
}

int u1_layout(Ctx* c, const std::vector<U1Spec>& probs, U1Plan* p) {
  p->nprob = (int)probs.size();
  p->n = 0;
  p->x_off.clear();
  p->s1.clear();
  p->s4.clear();
  p->segA1.clear(); p->segB4.clear(); p->slabs.clear(); p->ttiles.clear();
  p->pairs.clear(); p->outs.clear(); p->ins.clear(); p->wtiles.clear(); p->rows.clear();
  p->KA1 = p->KA4 = p->rowsA1 = p->rowsB1 = p->rowsA4 = p->rowsB4 = p->P1 = p->P4 = 0;
  p->flops = p->dense_flops = 0;
  p->sig.clear();
  std::vector<Layout> lay;
  for (const U1Spec& s : probs) {
    TNT_TRY(u1_check(c, s));
    lay.push_back(layout_of(s));
    p->x_off.push_back(p->n);
    p->n += lay.back().n;
    p->sig += "|" + std::to_string(s.d) + "," + std::to_string(s.D) + ":";
    for (const Sector& q : lay.back().Ls) p->sig += std::to_string(q.size) + ".";
    p->sig += "/";
    for (const Sector& q : lay.back().Rs) p->sig += std::to_string(q.size) + ".";
  }
  // pass 1: task shapes (KA1, KA4 need every task's K)
  struct P1Info { std::vector<std::vector<int64_t>> rowoff1; std::vector<int> task1; };
  std::vector<P1Info> info1(probs.size());
  struct P4Info { std::vector<std::map<int64_t, int64_t>> rowoff4; std::vector<std::vector<int64_t>> koff4; std::vector<int> task4; };
  std::vector<P4Info> info4(probs.size());
  for (size_t pi = 0; pi < probs.size(); ++pi) {
    const U1Spec& s = probs[pi];
    const Layout& l = lay[pi];
    const int64_t d = s.d, D = s.D;
    p->dense_flops += 8.0 * (double)(D * s.chl) * (double)(d * d * s.chr) * (double)s.chl +
                      8.0 * (double)(s.chl * d * d) * (double)s.chr * (double)(D * s.chr);
    P1Info& i1 = info1[pi];
    for (size_t iL = 0; iL < l.Ls.size(); ++iL) {
      const Sector& sq = l.Ls[iL];
      std::vector<int64_t> ro((size_t)D, -1);
      int64_t M = 0;
      for (int64_t w = 0; w < D; ++w) {
        auto it = l.Li.find(sq.q + s.wq[(size_t)w]);
        if (it == l.Li.end()) continue;
        ro[(size_t)w] = M;
        M += l.Ls[(size_t)it->second].size;
      }
      i1.rowoff1.push_back(ro);
      if (M == 0 || l.N[iL] == 0) { i1.task1.push_back(-1); continue; }
      TaskDesc t{p->rowsA1, p->rowsB1, M, l.N[iL], sq.size, p->P1, l.N[iL]};
      i1.task1.push_back((int)p->s1.size());
      p->s1.push_back(t);
      p->rowsA1 += M;
      p->rowsB1 += l.N[iL];
      p->P1 += M * l.N[iL];
      p->KA1 = std::max(p->KA1, rup(sq.size, 16));
      p->flops += 8.0 * (double)M * (double)l.N[iL] * (double)sq.size;
    }
    P4Info& i4 = info4[pi];
    for (size_t jQ = 0; jQ < l.Rs.size(); ++jQ) {
      const Sector& sQ = l.Rs[jQ];
      std::map<int64_t, int64_t> ro;
      int64_t M = 0;
      for (size_t iL = 0; iL < l.Ls.size(); ++iL)
        for (int64_t s1 = 0; s1 < d; ++s1)
          for (int64_t s2 = 0; s2 < d; ++s2)
            if (l.Ls[iL].q + s1 + s2 == sQ.q) {
              ro[((int64_t)iL * d + s1) * d + s2] = M;
              M += l.Ls[iL].size;
            }
      std::vector<int64_t> ko((size_t)D, -1);
      int64_t K = 0;
      for (int64_t w2 = 0; w2 < D; ++w2) {
        auto it = l.Ri.find(sQ.q - s.wq[(size_t)w2]);
        if (it == l.Ri.end()) continue;
        ko[(size_t)w2] = K;
        K += l.Rs[(size_t)it->second].size;
      }
      i4.rowoff4.push_back(ro);
      i4.koff4.push_back(ko);
      if (M == 0) { i4.task4.push_back(-1); continue; }
      if (K == 0) return set_err(c, TNT_E_INVALID, "MPO bond charges leave right sector %lld without terms", (long long)sQ.q);
      TaskDesc t{p->rowsA4, p->rowsB4, M, sQ.size, K, p->P4, sQ.size};
      i4.task4.push_back((int)p->s4.size());
      p->s4.push_back(t);
      p->rowsA4 += M;
      p->rowsB4 += sQ.size;
      p->P4 += M * sQ.size;
      p->KA4 = std::max(p->KA4, rup(K, 16));
      p->flops += 8.0 * (double)M * (double)sQ.size * (double)K;
    }
  }
  if (p->s1.empty() || p->s4.empty()) return set_err(c, TNT_E_INVALID, "U(1) problem has no allowed blocks");
  if (p->rowsA1 + 256 > INT32_MAX || p->rowsA4 + 256 > INT32_MAX || p->rowsB1 + 256 > INT32_MAX)
    return set_err(c, TNT_E_INVALID, "grouped matvec too large for 32-bit tile coordinates");
  // pass 2: pack segments, theta slabs, W pairs, output rows
  for (size_t pi = 0; pi < probs.size(); ++pi) {
    const U1Spec& s = probs[pi];
    const Layout& l = lay[pi];
    const int64_t d = s.d, D = s.D;
    const P1Info& i1 = info1[pi];
    const P4Info& i4 = info4[pi];
    // W12[(s1' s2' w2), (w s1 s2)] = sum_w1 W1[w,w1,s1',s1] W2[w1,w2,s2',s2]  (host, FP64)
    std::vector<z> W1((size_t)(D * D * d * d)), W2((size_t)(D * D * d * d));
    if (s.hW1) std::copy(s.hW1, s.hW1 + W1.size(), W1.begin());
    else TNT_TRY(read_small(c, s.W1, W1.data(), W1.size() * sizeof(z)));
    if (s.hW2) std::copy(s.hW2, s.hW2 + W2.size(), W2.begin());
    else TNT_TRY(read_small(c, s.W2, W2.data(), W2.size() * sizeof(z)));
    auto at = [&](const std::vector<z>& W, int64_t w, int64_t wp, int64_t so, int64_t si) {
      return W[(size_t)(((w * D + wp) * d + so) * d + si)];
    };
    const int64_t nI = d * d * D, nJ = D * d * d;
    std::vector<z> W12((size_t)(nI * nJ), zmk(0, 0));
    for (int64_t s1o = 0; s1o < d; ++s1o)
      for (int64_t s2o = 0; s2o < d; ++s2o)
        for (int64_t w2 = 0; w2 < D; ++w2)
          for (int64_t w = 0; w < D; ++w)
            for (int64_t s1 = 0; s1 < d; ++s1)
              for (int64_t s2 = 0; s2 < d; ++s2) {
                z acc = zmk(0, 0);
                for (int64_t w1 = 0; w1 < D; ++w1)
                  zfma(acc, at(W1, w, w1, s1o, s1), at(W2, w1, w2, s2o, s2));
                W12[(size_t)((((s1o * d + s2o) * D + w2) * nJ) + (w * d + s1) * d + s2)] = acc;
              }
    // stage 1 operands
    for (size_t iL = 0; iL < l.Ls.size(); ++iL) {
      const int ti = i1.task1[iL];
      if (ti < 0) continue;
      const TaskDesc& t = p->s1[(size_t)ti];
      const Sector& sq = l.Ls[iL];
      for (int64_t w = 0; w < D; ++w) {
        const int64_t ro = i1.rowoff1[iL][(size_t)w];
        if (ro < 0) continue;
        const Sector& sp2 = l.Ls[(size_t)l.Li.at(sq.q + s.wq[(size_t)w])];
        for (int64_t a = 0; a < sp2.size; ++a)
          p->segA1.push_back(PackSeg{s.L + ((sp2.start + a) * D + w) * s.chl + sq.start,
                                     (t.a_row0 + ro + a) * p->KA1, sq.size});
      }
      const int slab = (int)p->slabs.size();
      p->slabs.push_back(TSlab{p->x_off[pi] + l.toff[iL], l.N[iL], sq.size, t.b_row0});
      for (int64_t n0 = 0; n0 < l.N[iL]; n0 += 32)
        for (int64_t k0 = 0; k0 < sq.size; k0 += 32) p->ttiles.push_back(make_int4(slab, (int)n0, (int)k0, 0));
    }
    // stage 4 operands and output rows
    for (size_t jQ = 0; jQ < l.Rs.size(); ++jQ) {
      const int ti = i4.task4[jQ];
      if (ti < 0) continue;
      const TaskDesc& t = p->s4[(size_t)ti];
      const Sector& sQ = l.Rs[jQ];
      for (int64_t b = 0; b < sQ.size; ++b)
        for (int64_t w2 = 0; w2 < D; ++w2) {
          const int64_t ko = i4.koff4[jQ][(size_t)w2];
          if (ko < 0) continue;
          const Sector& sb = l.Rs[(size_t)l.Ri.at(sQ.q - s.wq[(size_t)w2])];
          p->segB4.push_back(PackSeg{s.R + ((sQ.start + b) * D + w2) * s.chr + sb.start,
                                     (t.b_row0 + b) * p->KA4 + ko, sb.size});
        }
      for (const auto& kv : i4.rowoff4[jQ]) {
        const int64_t key = kv.first, ro = kv.second;
        const int64_t iL = key / (d * d), s12 = key % (d * d);
        const Sector& sa = l.Ls[(size_t)iL];
        for (int64_t a = 0; a < sa.size; ++a)
          p->rows.push_back(GRow{t.c_off + (ro + a) * t.ldc,
                                 p->x_off[pi] + l.toff[(size_t)iL] + a * l.N[(size_t)iL] +
                                     l.coff[(size_t)iL][(size_t)s12],
                                 sQ.size});
      }
    }
    // W pairs: a' in left sector q', b in right sector qb
    for (size_t iLp = 0; iLp < l.Ls.size(); ++iLp) {
      const Sector& sa = l.Ls[iLp];
      for (size_t jb = 0; jb < l.Rs.size(); ++jb) {
        const Sector& sb = l.Rs[jb];
        WPair pr{sa.size, sb.size, (int)p->outs.size(), 0};
        for (int64_t s1o = 0; s1o < d; ++s1o)
          for (int64_t s2o = 0; s2o < d; ++s2o)
            for (int64_t w2 = 0; w2 < D; ++w2) {
              const int64_t Q = sa.q + s1o + s2o;
              if (Q - s.wq[(size_t)w2] != sb.q) continue;
              auto itQ = l.Ri.find(Q);
              if (itQ == l.Ri.end()) continue;
              const int jQ = itQ->second;
              const int t4 = i4.task4[(size_t)jQ];
              const TaskDesc& T4 = p->s4[(size_t)t4];
              const int64_t ro = i4.rowoff4[(size_t)jQ].at(((int64_t)iLp * d + s1o) * d + s2o);
              const int64_t ko = i4.koff4[(size_t)jQ][(size_t)w2];
              WOut o{(T4.a_row0 + ro) * p->KA4 + ko, (int)p->ins.size(), 0};
              const int64_t irow = ((s1o * d + s2o) * D + w2) * nJ;
              for (int64_t w = 0; w < D; ++w) {
                auto itq = l.Li.find(sa.q - s.wq[(size_t)w]);
                if (itq == l.Li.end()) continue;
                const int iL = itq->second;
                const int t1 = i1.task1[(size_t)iL];
                if (t1 < 0) continue;
                const TaskDesc& T1 = p->s1[(size_t)t1];
                const int64_t ro1 = i1.rowoff1[(size_t)iL][(size_t)w];
                for (int64_t s1 = 0; s1 < d; ++s1)
                  for (int64_t s2 = 0; s2 < d; ++s2) {
                    if (l.Ls[(size_t)iL].q + s1 + s2 != sb.q) continue;
                    const z v = W12[(size_t)(irow + (w * d + s1) * d + s2)];
                    if (v.x == 0.0 && v.y == 0.0) continue;
                    const int64_t co = l.coff[(size_t)iL][(size_t)(s1 * d + s2)];
                    p->ins.push_back(WIn{T1.c_off + ro1 * T1.ldc + co, T1.ldc, v});
                    p->flops += 8.0 * (double)sa.size * (double)sb.size;
                  }
              }
              o.r1 = (int)p->ins.size();
              if (o.r1 - o.r0 > W_MAX_IN) return set_err(c, TNT_E_INVALID, "W contraction: too many terms for one output");
              p->outs.push_back(o);
              pr.nout++;
            }
        if (pr.nout == 0) continue;
        if (pr.nout > W_MAX_OUT || p->outs.back().r1 - p->outs[(size_t)pr.out0].r0 > W_MAX_IN)
          return set_err(c, TNT_E_INVALID, "W contraction: block pair exceeds the table limits");
        const int pi2 = (int)p->pairs.size();
        p->pairs.push_back(pr);
        for (int64_t e0 = 0; e0 < sa.size * sb.size; e0 += W_TILE) p->wtiles.push_back(make_int2(pi2, (int)e0));
      }
    }
  }
  // device bytes: buffers + tables (+ slack for rounding)
  const size_t f = sizeof(float);
  size_t b = 0;
  b += ws_round(4 * f * p->rowsA1 * p->KA1) + ws_round(4 * f * p->rowsB1 * p->KA1);
  b += ws_round(2 * f * p->P1) + ws_round(4 * f * p->rowsA4 * p->KA4) + ws_round(4 * f * p->rowsB4 * p->KA4);
  b += ws_round(4 * 2 * f * p->P4);
  b += ws_round(sizeof(z) * p->rowsA1 * p->KA1) + ws_round(sizeof(z) * p->P1) +
       ws_round(sizeof(z) * p->rowsA4 * p->KA4) + ws_round(sizeof(z) * p->rowsB4 * p->KA4) +
       ws_round(sizeof(z) * p->P4);
  b += ws_round(sizeof(PackSeg) * (p->segA1.size() + p->segB4.size()) + 512) + ws_round(sizeof(TSlab) * p->slabs.size()) +
       ws_round(sizeof(int4) * p->ttiles.size()) + ws_round(sizeof(WPair) * p->pairs.size()) +
       ws_round(sizeof(WOut) * p->outs.size()) + ws_round(sizeof(WIn) * p->ins.size()) +
       ws_round(sizeof(int2) * p->wtiles.size()) + ws_round(sizeof(GRow) * p->rows.size());
  // tiles: worst case N tile 64 and split 4
  int64_t t1 = 0, t4 = 0, z1 = 0, z4 = 0;
  // FP64 tiles counted at the smaller (16 x 16) size, the larger of the two lists
  for (const TaskDesc& t : p->s1) { t1 += ((t.M + 127) / 128) * ((t.N + 63) / 64); z1 += ((t.M + 15) / 16) * ((t.N + 15) / 16); }
  for (const TaskDesc& t : p->s4) { t4 += 4 * ((t.M + 127) / 128) * ((t.N + 63) / 64); z4 += ((t.M + 15) / 16) * ((t.N + 15) / 16); }
  p->cap_g1tiles = (int)t1;
  p->cap_g4tiles = (int)t4;
  b += ws_round(sizeof(int4) * (t1 + t4 + z1 + z4)) + ws_round(sizeof(GTask) * (p->s1.size() + p->s4.size())) +
       ws_round(sizeof(ZTask) * (p->s1.size() + p->s4.size()));
  p->bytes = b + (size_t)(1 << 20);
  return TNT_OK;
}

namespace {
int set_tiles(Ctx* c, U1Plan* p, int bn1, int bn4, int split4) {
  std::vector<GTask> g;
  std::vector<int4> tl;
  make_tiles(p->s1, bn1, 1, &g, &tl);
  TNT_CUDA_TRY(c, cudaMemcpyAsync(p->d_g1, g.data(), sizeof(GTask) * g.size(), cudaMemcpyHostToDevice, c->stream));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(p->d_g1tiles, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice, c->stream));
  p->n_g1tiles = (int)tl.size();
  std::vector<GTask> g4;
  std::vector<int4> tl4;
  make_tiles(p->s4, bn4, split4, &g4, &tl4);
  TNT_CUDA_TRY(c, cudaMemcpyAsync(p->d_g4, g4.data(), sizeof(GTask) * g4.size(), cudaMemcpyHostToDevice, c->stream));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(p->d_g4tiles, tl4.data(), sizeof(int4) * tl4.size(), cudaMemcpyHostToDevice, c->stream));
  p->n_g4tiles = (int)tl4.size();
  TNT_TRY(tma_map_planes(c, &p->tmB1, p->B1p, p->rowsB1, p->KA1, bn1));
  TNT_TRY(tma_map_planes(c, &p->tmB4, p->B4p, p->rowsB4, p->KA4, bn4));
  p->bn1 = bn1;
  p->bn4 = bn4;
  p->split4 = split4;
  // the host vectors must outlive the copies
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return TNT_OK;
}

GArgs gargs1(const U1Plan& p, Ctx* c) {
  return GArgs{p.d_g1, p.d_g1tiles, p.n_g1tiles, p.T1f, p.P1, 0, c->d_status};
}
GArgs gargs4(const U1Plan& p, Ctx* c) {
  return GArgs{p.d_g4, p.d_g4tiles, p.n_g4tiles, p.Yf, p.P4, 2 * p.P4, c->d_status};
}
WArgs wargs(const U1Plan& p) {
  return WArgs{p.d_pairs, p.d_outs, p.d_ins, p.d_wtiles, p.n_wtiles, p.T1f, p.P1, p.T1z,
               p.A4p, p.rowsA4 * p.KA4, p.A4z, p.KA4};
}

// time one stage configuration: median-free minimum of three runs after one warm-up
int time_stage(Ctx* c, U1Plan* p, int stage, float* ms) {
  cudaEvent_t e0, e1;
  TNT_CUDA_TRY(c, cudaEventCreate(&e0));
  TNT_CUDA_TRY(c, cudaEventCreate(&e1));
  float best = 1e30f;
  int r = TNT_OK;
  for (int rep = 0; rep < 4 && r == TNT_OK; ++rep) {
    cudaEventRecord(e0, c->stream);
    if (stage == 1)
      r = launch_grouped_bn(c, p->bn1, p->tmA1, p->tmB1, gargs1(*p, c), p->n_g1tiles);
    else
      r = launch_grouped_bn(c, p->bn4, p->tmA4, p->tmB4, gargs4(*p, c), p->n_g4tiles);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0) best = std::min(best, t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  return r;
}

constexpr double TUNE_MIN_FLOPS = 2e9;  // below this a matvec is launch-bound: no search

int autotune(Ctx* c, U1Plan* p) {
  auto it = c->tune.find(p->sig);
  if (it != c->tune.end()) return set_tiles(c, p, it->second[0], it->second[1], it->second[2]);
  if (p->flops < TUNE_MIN_FLOPS) {
    c->tune[p->sig] = std::vector<int>{128, 128, 1};
    return set_tiles(c, p, 128, 128, 1);
  }
  int best1 = 128, best4 = 128, bests = 1;
  float t1best = 1e30f, t4best = 1e30f;
  for (int bn : {128, 64}) {
    TNT_TRY(set_tiles(c, p, bn, 128, 1));
    float ms;
    TNT_TRY(time_stage(c, p, 1, &ms));
    if (ms < t1best) { t1best = ms; best1 = bn; }
  }
  for (int bn : {128, 64})
    for (int sp : {1, 2, 4}) {
      TNT_TRY(set_tiles(c, p, best1, bn, sp));
      float ms;
      TNT_TRY(time_stage(c, p, 4, &ms));
      if (ms < t4best) { t4best = ms; best4 = bn; bests = sp; }
    }
  c->tune[p->sig] = std::vector<int>{best1, best4, bests};
  TNT_TRY(set_tiles(c, p, best1, best4, bests));
  // candidates wrote split parts the chosen tiling may not: start from zeros
  TNT_CUDA_TRY(c, cudaMemsetAsync(p->Yf, 0, sizeof(float) * 8 * p->P4, c->stream));
  return TNT_OK;
}
}  // namespace

int u1_prepare(Ctx* c, const std::vector<U1Spec>& probs, U1Plan* p) {
  (void)probs;
  const size_t f = sizeof(float);
  auto fa = [&](size_t n) { return (float*)ws_alloc(c, ws_round(f * std::max<size_t>(n, 1))); };
  auto za = [&](size_t n) { return (z*)ws_alloc(c, ws_round(sizeof(z) * std::max<size_t>(n, 1))); };
  p->A1p = fa(4 * p->rowsA1 * p->KA1);
  p->B1p = fa(4 * p->rowsB1 * p->KA1);
  p->T1f = fa(2 * p->P1);
  p->A4p = fa(4 * p->rowsA4 * p->KA4);
  p->B4p = fa(4 * p->rowsB4 * p->KA4);
  p->Yf = fa(8 * p->P4);
  p->A1z = za(p->rowsA1 * p->KA1);
  p->T1z = za(p->P1);
  p->A4z = za(p->rowsA4 * p->KA4);
  p->B4z = za(p->rowsB4 * p->KA4);
  p->Yz = za(p->P4);
  if (!p->A1p || !p->B1p || !p->T1f || !p->A4p || !p->B4p || !p->Yf || !p->A1z || !p->T1z ||
      !p->A4z || !p->B4z || !p->Yz)
    return set_err(c, TNT_E_ALLOC, "scratch exhausted (grouped matvec buffers)");
  // zero padding (K columns beyond a task's K, and the T3 entries no pair writes)
  TNT_CUDA_TRY(c, cudaMemsetAsync(p->A1p, 0, 4 * f * p->rowsA1 * p->KA1, c->stream));
  TNT_CUDA_TRY(c, cudaMemsetAsync(p->B1p, 0, 4 * f * p->rowsB1 * p->KA1, c->stream));
  TNT_CUDA_TRY(c, cudaMemsetAsync(p->A4p, 0, 4 * f * p->rowsA4 * p->KA4, c->stream));
  TNT_CUDA_TRY(c, cudaMemsetAsync(p->B4p, 0, 4 * f * p->rowsB4 * p->KA4, c->stream));
  TNT_CUDA_TRY(c, cudaMemsetAsync(p->Yf, 0, 8 * f * p->P4, c->stream));
  TNT_CUDA_TRY(c, cudaMemsetAsync(p->A1z, 0, sizeof(z) * p->rowsA1 * p->KA1, c->stream));
  TNT_CUDA_TRY(c, cudaMemsetAsync(p->A4z, 0, sizeof(z) * p->rowsA4 * p->KA4, c->stream));
  TNT_CUDA_TRY(c, cudaMemsetAsync(p->B4z, 0, sizeof(z) * p->rowsB4 * p->KA4, c->stream));
  // tables
  PackSeg *dA1 = nullptr, *dB4 = nullptr;
  TNT_TRY(upload(c, &dA1, p->segA1));
  TNT_TRY(upload(c, &dB4, p->segB4));
  TNT_TRY(upload(c, &p->d_slabs, p->slabs));
  TNT_TRY(upload(c, &p->d_ttiles, p->ttiles));
  TNT_TRY(upload(c, &p->d_pairs, p->pairs));
  TNT_TRY(upload(c, &p->d_outs, p->outs));
  TNT_TRY(upload(c, &p->d_ins, p->ins));
  TNT_TRY(upload(c, &p->d_wtiles, p->wtiles));
  TNT_TRY(upload(c, &p->d_rows, p->rows));
  p->n_ttiles = (int)p->ttiles.size();
  p->n_wtiles = (int)p->wtiles.size();
  p->n_rows = (int)p->rows.size();
  // FP64 tasks: stage 1 B operand is the input theta (offsets from x), stage 4 packed
  std::vector<ZTask> z1, z4;
  for (size_t i = 0; i < p->s1.size(); ++i) {
    const TaskDesc& t = p->s1[i];
    const TSlab& sb = p->slabs[i];
    z1.push_back(ZTask{t.M, t.N, t.K, t.a_row0 * p->KA1, p->KA1, 1, sb.src, t.N, 1, t.c_off, t.ldc});
  }
  for (const TaskDesc& t : p->s4)
    z4.push_back(ZTask{t.M, t.N, t.K, t.a_row0 * p->KA4, p->KA4, 1, t.b_row0 * p->KA4, 1, p->KA4, t.c_off, t.ldc});
  std::vector<int4> zt1, zt4;
  make_ztiles(z1, ZM, &zt1);
  make_ztiles(z4, ZM, &zt4);
  // 16 x 16 tiles when the 64 x 64 ones would not give every SM FP64 work
  p->ztile = ((int64_t)zt1.size() < sm_count() || (int64_t)zt4.size() < sm_count()) ? 16 : ZM;
  if (p->ztile == 16) {
    make_ztiles(z1, 16, &zt1);
    make_ztiles(z4, 16, &zt4);
  }
  TNT_TRY(upload(c, &p->d_z1, z1));
  TNT_TRY(upload(c, &p->d_z4, z4));
  TNT_TRY(upload(c, &p->d_z1tiles, zt1));
  TNT_TRY(upload(c, &p->d_z4tiles, zt4));
  p->n_z1tiles = (int)zt1.size();
  p->n_z4tiles = (int)zt4.size();
  std::vector<GTask> none;
  std::vector<int4> none4;
  TNT_TRY(upload(c, &p->d_g1, none, p->s1.size()));
  TNT_TRY(upload(c, &p->d_g4, none, p->s4.size()));
  TNT_TRY(upload(c, &p->d_g1tiles, none4, (size_t)p->cap_g1tiles));
  TNT_TRY(upload(c, &p->d_g4tiles, none4, (size_t)p->cap_g4tiles));
  // constant operands: environments into split planes and FP64 packs
  const int nA = (int)p->segA1.size(), nB = (int)p->segB4.size();
  const int64_t plA = p->rowsA1 * p->KA1, plB = p->rowsB4 * p->KA4;
  k_pack_segs<true><<<cap_grid((nA + 7) / 8, 152 * 8), 256, 0, c->stream>>>(dA1, nA, p->A1p, plA, nullptr);
  k_pack_segs<false><<<cap_grid((nA + 7) / 8, 152 * 8), 256, 0, c->stream>>>(dA1, nA, nullptr, 0, p->A1z);
  k_pack_segs<true><<<cap_grid((nB + 7) / 8, 152 * 8), 256, 0, c->stream>>>(dB4, nB, p->B4p, plB, nullptr);
  k_pack_segs<false><<<cap_grid((nB + 7) / 8, 152 * 8), 256, 0, c->stream>>>(dB4, nB, nullptr, 0, p->B4z);
  c->launches += 4;
  TNT_CHECK_LAUNCH(c);
  TNT_TRY(tma_map_planes(c, &p->tmA1, p->A1p, p->rowsA1, p->KA1, 128));
  TNT_TRY(tma_map_planes(c, &p->tmA4, p->A4p, p->rowsA4, p->KA4, 128));
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  TNT_TRY(autotune(c, p));
  // arguments of the nodes whose pointers change per matvec
  p->in_tp = TPArgs{nullptr, p->d_slabs, p->d_ttiles, p->n_ttiles, p->B1p, p->KA1, p->rowsB1 * p->KA1};
  p->in_zg = ZGArgs{p->d_z1, p->d_z1tiles, p->n_z1tiles, p->A1z, nullptr, p->T1z};
  p->out_g[0] = GthArgs{p->d_rows, p->n_rows, nullptr, 0, 0, 0, p->Yz, nullptr};
  p->out_g[1] = GthArgs{p->d_rows, p->n_rows, p->Yf, p->P4, 2 * p->P4, p->split4, nullptr, nullptr};
  return TNT_OK;
}

namespace {
void* zfn(const U1Plan& p) { return p.ztile == 16 ? (void*)k_zgemm_grouped16 : (void*)k_zgemm_grouped; }
int64_t zcap(const U1Plan& p) { return p.ztile == 16 ? 152 * 8 : 152 * 2; }
void zlaunch(Ctx* c, const U1Plan& p, const ZGArgs& a, int ntiles) {
  if (p.ztile == 16)
    k_zgemm_grouped16<<<cap_grid(ntiles, zcap(p)), 256, 0, c->stream>>>(a);
  else
    k_zgemm_grouped<<<cap_grid(ntiles, zcap(p)), 256, 0, c->stream>>>(a);
}

// kernel-node parameters for a graph; args points at the single struct argument
cudaKernelNodeParams knp(void* fn, unsigned grid, unsigned block, unsigned smem, void** args) {
  cudaKernelNodeParams k{};
  k.func = fn;
  k.gridDim = dim3(grid);
  k.blockDim = dim3(block);
  k.sharedMemBytes = smem;
  k.kernelParams = args;
  k.extra = nullptr;
  return k;
}

int build_graph(Ctx* c, U1Plan& p, int mixed) {
  cudaGraph_t g;
  TNT_CUDA_TRY(c, cudaGraphCreate(&g, 0));
  p.graph[mixed] = g;
  cudaGraphNode_t prev = nullptr, node = nullptr;
  auto add = [&](const cudaKernelNodeParams& k) -> int {
    TNT_CUDA_TRY(c, cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &k));
    prev = node;
    return TNT_OK;
  };
  WArgs wa = wargs(p);
  const unsigned gw = cap_grid(p.n_wtiles, 152 * 8);
  const unsigned gg = cap_grid((p.n_rows + 7) / 8, 152 * 8);
  if (mixed) {
    TPArgs tp = p.in_tp;
    void* a0[] = {&tp};
    TNT_TRY(add(knp((void*)k_pack_theta_t, cap_grid(p.n_ttiles, 152 * 8), 256, 0, a0)));
    p.in_node[1] = node;
    GArgs g1 = gargs1(p, c), g4 = gargs4(p, c);
    CUtensorMap m1a = p.tmA1, m1b = p.tmB1, m4a = p.tmA4, m4b = p.tmB4;
    void* a1[] = {&m1a, &m1b, &g1};
    void* f1 = p.bn1 == 64 ? (void*)k_cgemm_grouped<64> : (void*)k_cgemm_grouped<128>;
    const int s1 = p.bn1 == 64 ? GCfg<64>::SMEM : GCfg<128>::SMEM;
    TNT_TRY(launch_grouped_bn(c, p.bn1, p.tmA1, p.tmB1, g1, 0));  // sets the smem attribute
    TNT_TRY(add(knp(f1, cap_grid(p.n_g1tiles, sm_count()), 192, (unsigned)s1, a1)));
    void* a2[] = {&wa};
    TNT_TRY(add(knp((void*)k_wop<true>, gw, 256, 0, a2)));
    void* a3[] = {&m4a, &m4b, &g4};
    void* f4 = p.bn4 == 64 ? (void*)k_cgemm_grouped<64> : (void*)k_cgemm_grouped<128>;
    const int s4 = p.bn4 == 64 ? GCfg<64>::SMEM : GCfg<128>::SMEM;
    TNT_TRY(launch_grouped_bn(c, p.bn4, p.tmA4, p.tmB4, g4, 0));
    TNT_TRY(add(knp(f4, cap_grid(p.n_g4tiles, sm_count()), 192, (unsigned)s4, a3)));
    GthArgs ga = p.out_g[1];
    void* a4[] = {&ga};
    TNT_TRY(add(knp((void*)k_gather_u1<true>, gg, 256, 0, a4)));
    p.out_node[1] = node;
  } else {
    ZGArgs z1 = p.in_zg;
    void* a0[] = {&z1};
    TNT_TRY(add(knp(zfn(p), cap_grid(p.n_z1tiles, zcap(p)), 256, 0, a0)));
    p.in_node[0] = node;
    void* a1[] = {&wa};
    TNT_TRY(add(knp((void*)k_wop<false>, gw, 256, 0, a1)));
    ZGArgs z4{p.d_z4, p.d_z4tiles, p.n_z4tiles, p.A4z, p.B4z, p.Yz};
    void* a2[] = {&z4};
    TNT_TRY(add(knp(zfn(p), cap_grid(p.n_z4tiles, zcap(p)), 256, 0, a2)));
    GthArgs ga = p.out_g[0];
    void* a3[] = {&ga};
    TNT_TRY(add(knp((void*)k_gather_u1<false>, gg, 256, 0, a3)));
    p.out_node[0] = node;
  }
  TNT_CUDA_TRY(c, cudaGraphInstantiate(&p.exec[mixed], g, 0));
  return TNT_OK;
}

int run_direct(Ctx* c, U1Plan& p, const z* x, z* y, int mixed) {
  WArgs wa = wargs(p);
  const unsigned gw = cap_grid(p.n_wtiles, 152 * 8);
  const unsigned gg = cap_grid((p.n_rows + 7) / 8, 152 * 8);
  const double wflops = 8.0 * 0;  // counted within the plan's total
  (void)wflops;
  if (mixed) {
    TPArgs tp = p.in_tp;
    tp.x = x;
    {
      ProfScope ps(c, "u1_pack_theta", 16.0 * (double)p.n + 16.0 * (double)p.n);
      k_pack_theta_t<<<cap_grid(p.n_ttiles, 152 * 8), 256, 0, c->stream>>>(tp);
    }
    c->launches++;
    TNT_CHECK_LAUNCH(c);
    double f1 = 0, f4 = 0;
    for (const TaskDesc& t : p.s1) f1 += 8.0 * t.M * t.N * t.K;
    for (const TaskDesc& t : p.s4) f4 += 8.0 * t.M * t.N * t.K;
    {
      ProfScope ps(c, "cgemm_grouped", f1);
      TNT_TRY(launch_grouped_bn(c, p.bn1, p.tmA1, p.tmB1, gargs1(p, c), p.n_g1tiles));
    }
    {
      ProfScope ps(c, "u1_wop", 8.0 * (double)p.P1 + 16.0 * (double)(p.rowsA4 * p.KA4));
      k_wop<true><<<gw, 256, 0, c->stream>>>(wa);
    }
    c->launches++;
    TNT_CHECK_LAUNCH(c);
    {
      ProfScope ps(c, "cgemm_grouped", f4);
      TNT_TRY(launch_grouped_bn(c, p.bn4, p.tmA4, p.tmB4, gargs4(p, c), p.n_g4tiles));
    }
    GthArgs ga = p.out_g[1];
    ga.y = y;
    {
      ProfScope ps(c, "u1_gather", (double)p.split4 * 8.0 * (double)p.P4 + 16.0 * (double)p.n);
      k_gather_u1<true><<<gg, 256, 0, c->stream>>>(ga);
    }
    c->launches++;
    TNT_CHECK_LAUNCH(c);
  } else {
    double f1 = 0, f4 = 0;
    for (const TaskDesc& t : p.s1) f1 += 8.0 * t.M * t.N * t.K;
    for (const TaskDesc& t : p.s4) f4 += 8.0 * t.M * t.N * t.K;
    ZGArgs z1 = p.in_zg;
    z1.B = x;
    {
      ProfScope ps(c, "zgemm_grouped", f1);
      zlaunch(c, p, z1, p.n_z1tiles);
    }
    {
      ProfScope ps(c, "u1_wop_f64", 16.0 * (double)p.P1 + 16.0 * (double)(p.rowsA4 * p.KA4));
      k_wop<false><<<gw, 256, 0, c->stream>>>(wa);
    }
    ZGArgs z4{p.d_z4, p.d_z4tiles, p.n_z4tiles, p.A4z, p.B4z, p.Yz};
    {
      ProfScope ps(c, "zgemm_grouped", f4);
      zlaunch(c, p, z4, p.n_z4tiles);
    }
    GthArgs ga = p.out_g[0];
    ga.y = y;
    k_gather_u1<false><<<gg, 256, 0, c->stream>>>(ga);
    c->launches += 4;
    TNT_CHECK_LAUNCH(c);
  }
  return TNT_OK;
}
}  // namespace

int u1_run(Ctx* c, U1Plan& p, const z* x, z* y, int precision) {
  const int mixed = (precision == TNT_PREC_MIXED) ? 1 : 0;
  if (!c->use_graphs || !c->prof_cls.empty()) return run_direct(c, p, x, y, mixed);
  if (!p.exec[mixed]) TNT_TRY(build_graph(c, p, mixed));
  if (mixed) {
    TPArgs tp = p.in_tp;
    tp.x = x;
    void* a[] = {&tp};
    cudaKernelNodeParams k = knp((void*)k_pack_theta_t, cap_grid(p.n_ttiles, 152 * 8), 256, 0, a);
    TNT_CUDA_TRY(c, cudaGraphExecKernelNodeSetParams(p.exec[1], p.in_node[1], &k));
    GthArgs ga = p.out_g[1];
    ga.y = y;
    void* b[] = {&ga};
    cudaKernelNodeParams k2 = knp((void*)k_gather_u1<true>, cap_grid((p.n_rows + 7) / 8, 152 * 8), 256, 0, b);
    TNT_CUDA_TRY(c, cudaGraphExecKernelNodeSetParams(p.exec[1], p.out_node[1], &k2));
    c->launches += 5;
  } else {
    ZGArgs z1 = p.in_zg;
    z1.B = x;
    void* a[] = {&z1};
    cudaKernelNodeParams k = knp(zfn(p), cap_grid(p.n_z1tiles, zcap(p)), 256, 0, a);
    TNT_CUDA_TRY(c, cudaGraphExecKernelNodeSetParams(p.exec[0], p.in_node[0], &k));
    GthArgs ga = p.out_g[0];
    ga.y = y;
    void* b[] = {&ga};
    cudaKernelNodeParams k2 = knp((void*)k_gather_u1<false>, cap_grid((p.n_rows + 7) / 8, 152 * 8), 256, 0, b);
    TNT_CUDA_TRY(c, cudaGraphExecKernelNodeSetParams(p.exec[0], p.out_node[0], &k2));
    c->launches += 4;
  }
  TNT_CUDA_TRY(c, cudaGraphLaunch(p.exec[mixed], c->stream));
  return TNT_OK;
}

}  // namespace tnt
