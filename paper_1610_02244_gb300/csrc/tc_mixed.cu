// Split-TF32 tensor-core path of H_eff.theta (tcgen05 + TMA + TMEM, sm_103a).
//
// The two chi^3 contractions of the matvec (T1 = L.theta and y = T3.R^T, the GEMM steps of
// App. B.1.1 applied in the Listing 1 order) run as complex GEMMs C = A B^T on the 5th
// generation tensor cores.  Each FP64 operand x is split into TF32 parts
// hi = tf32(x), lo = tf32(x - hi) (22 significant bits together) and each complex product
// is accumulated in FP32 from three real products per part pair:
//   C_re += A_re^hi B_re^hi + A_re^hi B_re^lo + A_re^lo B_re^hi
//         - (A_im^hi B_im^hi + A_im^hi B_im^lo + A_im^lo B_im^hi)
//   C_im += A_re^hi B_im^hi + A_re^hi B_im^lo + A_re^lo B_im^hi
//         + A_im^hi B_re^hi + A_im^hi B_re^lo + A_im^lo B_re^hi
// (12 tcgen05.mma per k-block; the subtracted A_im B_im terms go to a third TMEM
// accumulator that the epilogue subtracts).  The W contraction between the two GEMMs,
// the reductions and the output stay FP64.
//
// CTA layout (192 threads): warp 0 = TMA producer, warp 1 = TMEM owner and MMA issuer
// (one elected thread), warps 2..5 = epilogue (TMEM lanes 32*(warp%4)..+31).
// Every mbarrier wait is bounded by %globaltimer; on expiry the CTA records an error in
// the context's status word, waits for its own copies, frees TMEM and returns.
#include <cmath>

#include "heff_plan.cuh"
#include "tc_common.cuh"

namespace tnt {

namespace {
using namespace tc;
constexpr int BM = 128, BN = 128, BK = 16;  // BK in FP32 elements: 64-byte rows
constexpr int STAGES = 3;
constexpr int TILE_A = BM * BK * 4;          // 8 KB per plane tile
constexpr int TILE_B = BN * BK * 4;
constexpr int STAGE_BYTES = 4 * TILE_A + 4 * TILE_B;   // 64 KB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int TMEM_COLS = 4 * BN;            // acc_re+ | acc_im | acc_re- | (unused): 512

struct CG {
  int64_t M, N;         // valid output extent
  int kb_total;         // k-blocks of BK
  int kb_per_split;
  float* C;             // [split][2][M][ldc]  (re plane, then im plane)
  int64_t ldc;
  int64_t plane;        // M * ldc
  int* status;
};

__global__ void __launch_bounds__(192, 1) k_cgemm_tf32x3(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmB,
                                                         CG g) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accb = empty + STAGES;
  uint32_t* tmem_slot = (uint32_t*)(accb + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb0 = blockIdx.z * g.kb_per_split;
  const int kb1 = min(g.kb_total, kb0 + g.kb_per_split);
  const int nkb = kb1 - kb0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accb, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer
    int issued = 0;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % STAGES;
      if (i >= STAGES && !mbar_wait(&empty[s], ((i / STAGES) & 1) ^ 1, g.status)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      uint8_t* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      const int k = (kb0 + i) * BK;
      for (int p = 0; p < 4; ++p) tma_load3(st + p * TILE_A, &tmA, &full[s], k, m0, p);
      for (int p = 0; p < 4; ++p) tma_load3(st + 4 * TILE_A + p * TILE_B, &tmB, &full[s], k, n0, p);
      issued = i + 1;
    }
    // drain: every stage this thread filled must have landed before the CTA may exit
    for (int i = (issued > STAGES ? issued - STAGES : 0); i < issued; ++i)
      mbar_wait(&full[i % STAGES], (i / STAGES) & 1, g.status);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issuer
    const uint32_t id = idesc_tf32_n(BN);
    const uint32_t t_re = tmem, t_im = tmem + BN, t_rn = tmem + 2 * BN;
    bool ok = true;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % STAGES;
      if (!mbar_wait(&full[s], (i / STAGES) & 1, g.status)) {
        *abort_flag = 1;
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = su32(smem + s * STAGE_BYTES);
      for (int ks = 0; ks < BK / 8; ++ks) {  // K = 8 per tf32 MMA: 32 bytes along the row
        const uint32_t off = ks * 32;
        const uint64_t a_rh = desc_sw64(base + 0 * TILE_A + off);
        const uint64_t a_rl = desc_sw64(base + 1 * TILE_A + off);
        const uint64_t a_ih = desc_sw64(base + 2 * TILE_A + off);
        const uint64_t a_il = desc_sw64(base + 3 * TILE_A + off);
        const uint32_t bb = base + 4 * TILE_A;
        const uint64_t b_rh = desc_sw64(bb + 0 * TILE_B + off);
        const uint64_t b_rl = desc_sw64(bb + 1 * TILE_B + off);
        const uint64_t b_ih = desc_sw64(bb + 2 * TILE_B + off);
        const uint64_t b_il = desc_sw64(bb + 3 * TILE_B + off);
        const uint32_t first = (i == 0 && ks == 0) ? 0u : 1u;
        // real part: re_re products (+) and im_im products (accumulated apart, subtracted)
        mma_tf32(t_re, a_rh, b_rh, id, first);
        mma_tf32(t_re, a_rh, b_rl, id, 1);
        mma_tf32(t_re, a_rl, b_rh, id, 1);
        mma_tf32(t_rn, a_ih, b_ih, id, first);
        mma_tf32(t_rn, a_ih, b_il, id, 1);
        mma_tf32(t_rn, a_il, b_ih, id, 1);
        // imaginary part
        mma_tf32(t_im, a_rh, b_ih, id, first);
        mma_tf32(t_im, a_rh, b_il, id, 1);
        mma_tf32(t_im, a_rl, b_ih, id, 1);
        mma_tf32(t_im, a_ih, b_rh, id, 1);
        mma_tf32(t_im, a_ih, b_rl, id, 1);
        mma_tf32(t_im, a_il, b_rh, id, 1);
      }
      mma_commit(&empty[s]);  // stage s is free once these MMAs have read it
    }
    (void)ok;
    mma_commit(accb);  // accumulators complete (arrives after all MMAs issued above)
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue: TMEM -> global (FP32)
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int row = q * 32 + lane;
    const bool ok = mbar_wait(accb, 0, g.status);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && !*abort_flag) {
      const int64_t gm = m0 + row;
      float* Cre = g.C + (int64_t)blockIdx.z * 2 * g.plane;
      float* Cim = Cre + g.plane;
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32], s[32], u[32];
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        tmem_ld32(tmem + lane_addr + c0, r);
        tmem_ld32(tmem + lane_addr + BN + c0, s);
        tmem_ld32(tmem + lane_addr + 2 * BN + c0, u);
        if (gm < g.M) {
          float* pr = Cre + gm * g.ldc + n0 + c0;
          float* pi = Cim + gm * g.ldc + n0 + c0;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (n0 + c0 + j < g.N) {
              pr[j] = __uint_as_float(r[j]) - __uint_as_float(u[j]);
              pi[j] = __uint_as_float(s[j]);
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// planes[p][r][k] (rows Mp, K Kp) from src[r * ld + k] (r < M, k < K), zeros elsewhere
__global__ void k_split_rows(const z* __restrict__ src, int64_t M, int64_t K, int64_t ld,
                             int64_t Mp, int64_t Kp, float* __restrict__ out) {
  const int64_t plane = Mp * Kp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < plane;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / Kp, k = e % Kp;
    float a = 0, b = 0, c = 0, d = 0;
    if (r < M && k < K) {
      const z v = src[r * ld + k];
      split_tf32(v.x, &a, &b);
      split_tf32(v.y, &c, &d);
    }
    out[e] = a;
    out[plane + e] = b;
    out[2 * plane + e] = c;
    out[3 * plane + e] = d;
  }
}

// planes[p][n][k] (rows Np, K Kp) from src[k * N + n] (k < K, n < N): transpose via smem
__global__ void k_split_transpose(const z* __restrict__ src, int64_t K, int64_t N, int64_t Np,
                                  int64_t Kp, float* __restrict__ out) {
  __shared__ z tile[32][33];
  const int64_t plane = Np * Kp;
  const int64_t k0 = (int64_t)blockIdx.y * 32, nb = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int j = ty; j < 32; j += 8) {
    const int64_t k = k0 + j, n = nb + tx;
    tile[j][tx] = (k < K && n < N) ? src[k * N + n] : zmk(0, 0);
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t n = nb + j, k = k0 + tx;
    if (n < Np && k < Kp) {
      const z v = tile[tx][j];
      float a, b, c, d;
      split_tf32(v.x, &a, &b);
      split_tf32(v.y, &c, &d);
      const int64_t e = n * Kp + k;
      out[e] = a;
      out[plane + e] = b;
      out[2 * plane + e] = c;
      out[3 * plane + e] = d;
    }
  }
}

// T3 planes = W12 (x) T1 (FP32 re/im planes in, split TF32 planes out).  FP32 arithmetic:
// T1 itself carries the split-TF32 products' ~2^-22 relative error and W12 has a handful of
// O(1) entries per output, so FP64 here would buy nothing (and ran on the FP64 pipe).
__global__ void __launch_bounds__(256) k_op_mixed(OpApply a, const float* __restrict__ t1,
                                                  int64_t t1_plane, float* __restrict__ t3,
                                                  int64_t t3_plane) {
  __shared__ int s_row[257];
  __shared__ int s_col[2048];
  __shared__ float2 s_val[2048];
  __shared__ int64_t s_in[256];
  __shared__ int64_t s_out[256];
  for (int t = threadIdx.x; t <= a.nI; t += blockDim.x) s_row[t] = a.row_ptr[t];
  for (int t = threadIdx.x; t < a.nnz; t += blockDim.x) {
    s_col[t] = a.col[t];
    s_val[t] = make_float2((float)a.val[t].x, (float)a.val[t].y);
  }
  for (int t = threadIdx.x; t < a.nJ; t += blockDim.x) s_in[t] = a.in_off[t];
  for (int t = threadIdx.x; t < a.nI; t += blockDim.x) s_out[t] = a.out_off[t];
  __syncthreads();
  const int64_t total = a.B0 * a.B2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b2 = e % a.B2, b0 = e / a.B2;
    const float* ire = t1 + b0 * a.is0 + b2 * a.is2;
    const float* iim = ire + t1_plane;
    float* o = t3 + b0 * a.os0 + b2 * a.os2;
    for (int i = 0; i < a.nI; ++i) {
      float xr = 0.f, xi = 0.f;
      for (int t = s_row[i]; t < s_row[i + 1]; ++t) {
        const float2 w = s_val[t];
        const int64_t off = s_in[s_col[t]];
        const float vr = ire[off], vi = iim[off];
        xr = fmaf(w.x, vr, fmaf(-w.y, vi, xr));
        xi = fmaf(w.x, vi, fmaf(w.y, vr, xi));
      }
      float h, l;
      const int64_t off = s_out[i];
      split_tf32(xr, &h, &l);
      o[off] = h;
      o[t3_plane + off] = l;
      split_tf32(xi, &h, &l);
      o[2 * t3_plane + off] = h;
      o[3 * t3_plane + off] = l;
    }
  }
}

// y (FP64 interleaved, M x N) = sum over splits of the FP32 (re, im) planes, fixed order
__global__ void k_gather_y(const float* __restrict__ Yp, int split, int64_t M, int64_t N,
                           z* __restrict__ y) {
  const int64_t plane = M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < plane;
       e += (int64_t)gridDim.x * blockDim.x) {
    // the split-K partials are FP32 sums of split-TF32 products (~2^-22): added in FP32,
    // widened once by integer operations (no FP64-pipe conversion in the loop)
    float re = 0.f, im = 0.f;
    for (int s = 0; s < split; ++s) {
      re += Yp[(int64_t)s * 2 * plane + e];
      im += Yp[(int64_t)s * 2 * plane + plane + e];
    }
    y[e] = zmk(f64_of(re), f64_of(im));
  }
}

unsigned grid1(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return (unsigned)b;
}
int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int get_encoder(Ctx* c, EncodeTiledFn* fn) {
  static EncodeTiledFn cached = nullptr;
  if (!cached) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    TNT_CUDA_TRY(c, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                     cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p)
      return set_err(c, TNT_E_CUDA, "cuTensorMapEncodeTiled not available from the driver");
    cached = (EncodeTiledFn)p;
  }
  *fn = cached;
  return TNT_OK;
}

// 3-D map over planes[nplanes][rows][K]: box = 16 FP32 (64 B) x box_rows x 1, 64-byte swizzle
int make_map(Ctx* c, CUtensorMap* tm, float* base, int64_t rows, int64_t K, int box_rows,
             int nplanes = 4) {
  EncodeTiledFn enc;
  TNT_TRY(get_encoder(c, &enc));
  if (((uintptr_t)base & 15) || (K * 4) % 16)
    return set_err(c, TNT_E_INVALID, "TMA operand not 16-byte aligned");
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)nplanes};
  cuuint64_t strides[2] = {(cuuint64_t)(K * 4), (cuuint64_t)(rows * K * 4)};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_err(c, TNT_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return TNT_OK;
}

int launch_cgemm(Ctx* c, const CUtensorMap& tA, const CUtensorMap& tB, int64_t M, int64_t N,
                 int64_t Kp, int split, float* C, int64_t ldc, int64_t K_true) {
  static bool attr = false;
  if (!attr) {
    TNT_CUDA_TRY(c, cudaFuncSetAttribute(k_cgemm_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_BYTES));
    attr = true;
  }
  CG g;
  g.M = M;
  g.N = N;
  g.kb_total = (int)(Kp / BK);
  g.kb_per_split = (g.kb_total + split - 1) / split;
  g.C = C;
  g.ldc = ldc;
  g.plane = M * ldc;
  g.status = c->d_status;
  // every split must own at least one k-block (its accumulator is otherwise unset)
  if ((int64_t)g.kb_per_split * (split - 1) >= g.kb_total)
    return set_err(c, TNT_E_INVALID, "split-K %d leaves an empty split", split);
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)split);
  ProfScope ps(c, "cgemm_tf32x3", 8.0 * (double)M * (double)N * (double)K_true);
  k_cgemm_tf32x3<<<grid, 192, SMEM_BYTES, c->stream>>>(tA, tB, g);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}
}  // namespace

int tma_map_planes(Ctx* c, CUtensorMap* tm, float* base, int64_t rows, int64_t K, int box_rows) {
  return make_map(c, tm, base, rows, K, box_rows);
}
int tma_map_planes_n(Ctx* c, CUtensorMap* tm, float* base, int64_t rows, int64_t K, int box_rows,
                     int nplanes) {
  return make_map(c, tm, base, rows, K, box_rows, nplanes);
}

size_t heff_mixed_scratch_bound(int64_t chl, int64_t d, int64_t D, int64_t chr) {
  const int64_t Mp1 = rup(chl * D, BM), Kp1 = rup(chl, BK), Np1 = rup(d * d * chr, BN);
  const int64_t M4 = chl * d * d, Mp4 = rup(M4, BM), Kp4 = rup(D * chr, BK), Np4 = rup(chr, BN);
  size_t b = 0;
  b += ws_round(4 * sizeof(float) * Mp1 * Kp1);
  b += ws_round(4 * sizeof(float) * Np1 * Kp1);
  b += ws_round(2 * sizeof(float) * chl * D * d * d * chr);
  b += ws_round(4 * sizeof(float) * Mp4 * Kp4);
  b += ws_round(4 * sizeof(float) * Np4 * Kp4);
  b += ws_round(4 * 2 * sizeof(float) * M4 * chr);
  return b + (1 << 20);
}

int heff_mixed_prepare(Ctx* c, HeffPlan* p) {
  MixedPlan& m = p->mixed;
  const int64_t chl = p->chl, d = p->d, D = p->D, chr = p->chr;
  m.M1 = chl * D;
  m.N1 = d * d * chr;
  m.K1 = chl;
  m.Mp1 = rup(m.M1, BM);
  m.Np1 = rup(m.N1, BN);
  m.Kp1 = rup(m.K1, BK);
  m.M4 = chl * d * d;
  m.N4 = chr;
  m.K4 = D * chr;
  m.Mp4 = rup(m.M4, BM);
  m.Np4 = rup(m.N4, BN);
  m.Kp4 = rup(m.K4, BK);
  // split-K for stage 4 so that about two CTAs per SM are in flight
  const int64_t tiles4 = (m.Mp4 / BM) * (m.Np4 / BN);
  const int kb4 = (int)(m.Kp4 / BK);
  int split = (int)std::max<int64_t>(1, std::min<int64_t>(4, (2 * 152) / std::max<int64_t>(tiles4, 1)));
  while (split > 1 && (int64_t)((kb4 + split - 1) / split) * (split - 1) >= kb4) --split;
  m.split4 = split;
  m.Lp = (float*)ws_alloc(c, ws_round(4 * sizeof(float) * m.Mp1 * m.Kp1));
  m.Thp = (float*)ws_alloc(c, ws_round(4 * sizeof(float) * m.Np1 * m.Kp1));
  m.T1 = (float*)ws_alloc(c, ws_round(2 * sizeof(float) * m.M1 * m.N1));
  m.T3p = (float*)ws_alloc(c, ws_round(4 * sizeof(float) * m.Mp4 * m.Kp4));
  m.Rp = (float*)ws_alloc(c, ws_round(4 * sizeof(float) * m.Np4 * m.Kp4));
  m.Yp = (float*)ws_alloc(c, ws_round((size_t)split * 2 * sizeof(float) * m.M4 * m.N4));
  if (!m.Lp || !m.Thp || !m.T1 || !m.T3p || !m.Rp || !m.Yp)
    return set_err(c, TNT_E_ALLOC, "scratch exhausted (mixed-precision operands)");
  // constant operands: L rows (a', w) x K = a;  R rows b' x K = (w2, b)
  k_split_rows<<<grid1(m.Mp1 * m.Kp1), 256, 0, c->stream>>>(p->L, m.M1, m.K1, chl, m.Mp1, m.Kp1, m.Lp);
  k_split_rows<<<grid1(m.Np4 * m.Kp4), 256, 0, c->stream>>>(p->R, m.N4, m.K4, D * chr, m.Np4, m.Kp4, m.Rp);
  c->launches += 2;
  TNT_CUDA_TRY(c, cudaMemsetAsync(m.T3p, 0, 4 * sizeof(float) * m.Mp4 * m.Kp4, c->stream));
  TNT_CHECK_LAUNCH(c);
  TNT_TRY(make_map(c, &m.tmL, m.Lp, m.Mp1, m.Kp1, BM));
  TNT_TRY(make_map(c, &m.tmTh, m.Thp, m.Np1, m.Kp1, BN));
  TNT_TRY(make_map(c, &m.tmT3, m.T3p, m.Mp4, m.Kp4, BM));
  TNT_TRY(make_map(c, &m.tmR, m.Rp, m.Np4, m.Kp4, BN));
  // W12 with output offsets in T3-plane units: row (a' s1' s2'), column (w2 b)
  m.op = p->op;
  const int nI = (int)(d * d * D);
  std::vector<int64_t> out_off(nI);
  for (int64_t s1 = 0; s1 < d; ++s1)
    for (int64_t s2 = 0; s2 < d; ++s2)
      for (int64_t w2 = 0; w2 < D; ++w2)
        out_off[(size_t)((s1 * d + s2) * D + w2)] = (s1 * d + s2) * m.Kp4 + w2 * chr;
  int64_t* d_out = (int64_t*)ws_alloc(c, ws_round(sizeof(int64_t) * nI));
  if (!d_out) return set_err(c, TNT_E_ALLOC, "scratch exhausted (mixed op table)");
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_out, out_off.data(), sizeof(int64_t) * nI, cudaMemcpyHostToDevice, c->stream));
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  m.op.out_off = d_out;
  m.op.B0 = chl;
  m.op.B1 = 1;
  m.op.B2 = chr;
  m.op.is0 = D * d * d * chr;  // T1 plane: row (a' w) of length N1 = d^2 chr
  m.op.is2 = 1;
  m.op.os0 = d * d * m.Kp4;    // T3 plane: d^2 rows of Kp4 per a'
  m.op.os2 = 1;
  return TNT_OK;
}

int heff_run_mixed(Ctx* c, const HeffPlan& p, const z* theta, z* y) {
  const MixedPlan& m = p.mixed;
  // theta[a][(s1 s2 b)] -> planes [(s1 s2 b)][a]
  dim3 gt((unsigned)((m.Np1 + 31) / 32), (unsigned)((m.Kp1 + 31) / 32));
  {
    ProfScope ps(c, "split_theta", 32.0 * (double)m.K1 * (double)m.N1);
    k_split_transpose<<<gt, 256, 0, c->stream>>>(theta, m.K1, m.N1, m.Np1, m.Kp1, m.Thp);
  }
  c->launches++;
  TNT_TRY(launch_cgemm(c, m.tmL, m.tmTh, m.M1, m.N1, m.Kp1, 1, m.T1, m.N1, m.K1));
  int64_t total = m.op.B0 * m.op.B2;
  int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
  {
    ProfScope ps(c, "op_mixed", 8.0 * (double)m.M1 * (double)m.N1 + 16.0 * (double)m.M4 * (double)m.K4);
    k_op_mixed<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, c->stream>>>(
        m.op, m.T1, m.M1 * m.N1, m.T3p, m.Mp4 * m.Kp4);
  }
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  TNT_TRY(launch_cgemm(c, m.tmT3, m.tmR, m.M4, m.N4, m.Kp4, m.split4, m.Yp, m.N4, m.K4));
  k_gather_y<<<grid1(m.M4 * m.N4), 256, 0, c->stream>>>(m.Yp, m.split4, m.M4, m.N4, y);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

}  // namespace tnt
