// FP64 building blocks of the two-site update: strided complex GEMM (the contraction
// primitive of App. B.1.1: reorder indices, one matrix product -- here the reorder is
// folded into the strides), a sparse small-operator kernel for the MPO and gate legs,
// the Lanczos vector operations and the tridiagonal eigensolve.
#include <cstdarg>
#include <cmath>

#include "tnt_internal.cuh"
#include "f32conv.cuh"

namespace tnt {

// ============================================================ complex FP64 GEMM
// 64x64 output tile, BK = 16, 256 threads as 16x16; thread (tx, ty) owns rows ty + 16 r
// and columns tx + 16 c (r, c < 4) so stores are coalesced along the row.
namespace {
constexpr int GM = 64, GN = 64, GK = 16;

__global__ void __launch_bounds__(256) k_zgemm(ZGemm g) {
  __shared__ z As[GK][GM + 1];
  __shared__ z Bs[GK][GN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * GM, n0 = (int64_t)blockIdx.x * GN;
  if (g.lower_only && m0 + GM <= n0) return;  // strictly upper tile of a Hermitian result
  const int64_t bt = blockIdx.z;
  const z* A = g.A + bt * g.a_bs;
  const z* B = g.B + bt * g.b_bs;
  z* C = g.C + bt * g.c_bs;
  z acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = zmk(0, 0);
  const bool a_kfast = (g.a_cs == 1);
  const bool b_nfast = (g.b_cs == 1);
  for (int64_t k0 = 0; k0 < g.K; k0 += GK) {
#pragma unroll
    for (int t = 0; t < (GM * GK) / 256; ++t) {
      int e = threadIdx.x + 256 * t;
      int i, k;
      if (a_kfast) { k = e % GK; i = e / GK; } else { i = e % GM; k = e / GM; }
      int64_t gi = m0 + i, gk = k0 + k;
      z v = zmk(0, 0);
      if (gi < g.M && gk < g.K) {
        v = A[gi * g.a_rs + gk * g.a_cs];
        if (g.conj_a) v.y = -v.y;
      }
      As[k][i] = v;
    }
#pragma unroll
    for (int t = 0; t < (GN * GK) / 256; ++t) {
      int e = threadIdx.x + 256 * t;
      int j, k;
      if (b_nfast) { j = e % GN; k = e / GN; } else { k = e % GK; j = e / GK; }
      int64_t gj = n0 + j, gk = k0 + k;
      z v = zmk(0, 0);
      if (gj < g.N && gk < g.K) {
        v = B[gk * g.b_rs + gj * g.b_cs];
        if (g.conj_b) v.y = -v.y;
      }
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      z a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) zfma(acc[r][c], a[r], b[c]);
    }
    __syncthreads();
  }
  const bool use_beta = (g.beta.x != 0.0 || g.beta.y != 0.0);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int64_t gi = m0 + ty + 16 * r;
    if (gi >= g.M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int64_t gj = n0 + tx + 16 * c;
      if (gj >= g.N) continue;
      z v = zmul(g.alpha, acc[r][c]);
      z* p = C + gi * g.c_rs + gj;
      if (use_beta) v = zadd(v, zmul(g.beta, *p));
      *p = v;
    }
  }
}
}  // namespace

namespace {
// 16 x 16 output tiles, one element per thread: for products too small to give every SM
// a 64 x 64 tile (GB300's FP64 units are ~2 FMA per clock per SM, so the FP64 work of a
// small product must be spread thin)
__global__ void __launch_bounds__(256) k_zgemm16(ZGemm g) {
  __shared__ z As[16][17];
  __shared__ z Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * 16, n0 = (int64_t)blockIdx.x * 16;
  if (g.lower_only && m0 + 16 <= n0) return;
  const int64_t bt = blockIdx.z;
  const z* A = g.A + bt * g.a_bs;
  const z* B = g.B + bt * g.b_bs;
  z* C = g.C + bt * g.c_bs;
  z acc = zmk(0, 0);
  for (int64_t k0 = 0; k0 < g.K; k0 += 16) {
    {
      const int64_t gi = m0 + ty, gk = k0 + tx;
      z v = zmk(0, 0);
      if (gi < g.M && gk < g.K) {
        v = A[gi * g.a_rs + gk * g.a_cs];
        if (g.conj_a) v.y = -v.y;
      }
      As[ty][tx] = v;
    }
    {
      const int64_t gk = k0 + ty, gj = n0 + tx;
      z v = zmk(0, 0);
      if (gj < g.N && gk < g.K) {
        v = B[gk * g.b_rs + gj * g.b_cs];
        if (g.conj_b) v.y = -v.y;
      }
      Bs[ty][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) zfma(acc, As[ty][kk], Bs[kk][tx]);
    __syncthreads();
  }
  const int64_t gi = m0 + ty, gj = n0 + tx;
  if (gi < g.M && gj < g.N) {
    z v = zmul(g.alpha, acc);
    z* p = C + gi * g.c_rs + gj;
    if (g.beta.x != 0.0 || g.beta.y != 0.0) v = zadd(v, zmul(g.beta, *p));
    *p = v;
  }
}
}  // namespace

int zgemm(Ctx* c, const ZGemm& g) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return TNT_OK;
  if (g.K <= 0) {
    // C = beta C (or zero): not needed by the library; reject to keep the kernel simple
    return set_err(c, TNT_E_INVALID, "zgemm with K = 0");
  }
  if (ozgemm_eligible(c, g)) return ozgemm(c, g);
  {
    static int nsm = 0;
    if (!nsm && (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || nsm < 1))
      nsm = 152;
    const int64_t tiles64 = ((g.M + GM - 1) / GM) * ((g.N + GN - 1) / GN) * g.batch;
    if (tiles64 < nsm && (g.M + 15) / 16 <= 65535 && g.batch <= 65535) {
      dim3 grid((unsigned)((g.N + 15) / 16), (unsigned)((g.M + 15) / 16), (unsigned)g.batch);
      ProfScope ps(c, "zgemm_f64", (g.lower_only ? 4.0 : 8.0) * (double)g.M * (double)g.N *
                                       (double)g.K * (double)g.batch);
      k_zgemm16<<<grid, 256, 0, c->stream>>>(g);
      c->launches++;
      TNT_CHECK_LAUNCH(c);
      return TNT_OK;
    }
  }
  if ((g.N + GN - 1) / GN > 0x7fffffff || (g.M + GM - 1) / GM > 65535 || g.batch > 65535)
    return set_err(c, TNT_E_UNSUPPORTED, "zgemm grid too large (M=%lld N=%lld batch=%lld)",
                   (long long)g.M, (long long)g.N, (long long)g.batch);
  dim3 grid((unsigned)((g.N + GN - 1) / GN), (unsigned)((g.M + GM - 1) / GM),
            (unsigned)g.batch);
  ProfScope ps(c, "zgemm_f64", (g.lower_only ? 4.0 : 8.0) * (double)g.M * (double)g.N *
                                   (double)g.K * (double)g.batch);
  k_zgemm<<<grid, 256, 0, c->stream>>>(g);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

namespace {
__global__ void k_herm_mirror(z* G, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    if (i < j) G[e] = zconj(G[j * n + i]);
  }
}
}  // namespace

int herm_mirror(Ctx* c, z* G, int64_t n) {
  if (n <= 1) return TNT_OK;
  int64_t b = (n * n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  k_herm_mirror<<<(unsigned)b, 256, 0, c->stream>>>(G, n);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

// ============================================================ sparse operator apply
namespace {
constexpr int OP_MAX_NNZ = 2048;
constexpr int OP_MAX_LEG = 256;

__global__ void __launch_bounds__(256) k_op_apply(OpApply a, int nnz) {
  __shared__ int s_row[OP_MAX_LEG + 1];
  __shared__ int s_col[OP_MAX_NNZ];
  __shared__ z s_val[OP_MAX_NNZ];
  __shared__ int64_t s_in[OP_MAX_LEG];
  __shared__ int64_t s_out[OP_MAX_LEG];
  for (int t = threadIdx.x; t <= a.nI; t += blockDim.x) s_row[t] = a.row_ptr[t];
  for (int t = threadIdx.x; t < nnz; t += blockDim.x) {
    s_col[t] = a.col[t];
    s_val[t] = a.val[t];
  }
  for (int t = threadIdx.x; t < a.nJ; t += blockDim.x) s_in[t] = a.in_off[t];
  for (int t = threadIdx.x; t < a.nI; t += blockDim.x) s_out[t] = a.out_off[t];
  __syncthreads();
  const int64_t total = a.B0 * a.B1 * a.B2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t b2 = e % a.B2;
    int64_t r = e / a.B2;
    int64_t b1 = r % a.B1;
    int64_t b0 = r / a.B1;
    const z* in = a.in + b0 * a.is0 + b1 * a.is1 + b2 * a.is2;
    z* out = a.out + b0 * a.os0 + b1 * a.os1 + b2 * a.os2;
    for (int i = 0; i < a.nI; ++i) {
      z acc = zmk(0, 0);
      for (int t = s_row[i]; t < s_row[i + 1]; ++t) zfma(acc, s_val[t], in[s_in[s_col[t]]]);
      z* p = out + s_out[i];
      if (a.accumulate) acc = zadd(acc, *p);
      *p = acc;
    }
  }
}
}  // namespace

int op_upload(Ctx* c, const std::vector<z>& dense, int nI, int nJ,
              const std::vector<int64_t>& in_off, const std::vector<int64_t>& out_off,
              OpApply* a) {
  if (nI > OP_MAX_LEG || nJ > OP_MAX_LEG)
    return set_err(c, TNT_E_UNSUPPORTED, "operator legs %d x %d exceed %d", nI, nJ,
                   OP_MAX_LEG);
  std::vector<int> row(nI + 1, 0), col;
  std::vector<z> val;
  for (int i = 0; i < nI; ++i) {
    for (int j = 0; j < nJ; ++j) {
      z v = dense[(size_t)i * nJ + j];
      if (v.x != 0.0 || v.y != 0.0) {
        col.push_back(j);
        val.push_back(v);
      }
    }
    row[i + 1] = (int)col.size();
  }
  if (col.size() > (size_t)OP_MAX_NNZ)
    return set_err(c, TNT_E_UNSUPPORTED, "operator has %zu nonzeros > %d", col.size(),
                   OP_MAX_NNZ);
  if (col.empty()) {  // keep valid pointers for the kernel
    col.push_back(0);
    val.push_back(zmk(0, 0));
  }
  // one contiguous scratch block for the five tables
  size_t b_row = ws_round(sizeof(int) * row.size());
  size_t b_col = ws_round(sizeof(int) * col.size());
  size_t b_val = ws_round(sizeof(z) * val.size());
  size_t b_in = ws_round(sizeof(int64_t) * nJ);
  size_t b_out = ws_round(sizeof(int64_t) * nI);
  size_t total = b_row + b_col + b_val + b_in + b_out;
  char* dev = (char*)ws_alloc(c, total);
  if (!dev) return set_err(c, TNT_E_ALLOC, "scratch exhausted for operator tables");
  std::vector<char> host(total, 0);
  memcpy(host.data(), row.data(), sizeof(int) * row.size());
  memcpy(host.data() + b_row, col.data(), sizeof(int) * col.size());
  memcpy(host.data() + b_row + b_col, val.data(), sizeof(z) * val.size());
  memcpy(host.data() + b_row + b_col + b_val, in_off.data(), sizeof(int64_t) * nJ);
  memcpy(host.data() + b_row + b_col + b_val + b_in, out_off.data(), sizeof(int64_t) * nI);
  // synchronous: the host vector dies at return (tables are a few KB)
  TNT_CUDA_TRY(c, cudaMemcpyAsync(dev, host.data(), total, cudaMemcpyHostToDevice, c->stream));
  TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  a->nI = nI;
  a->nJ = nJ;
  a->nnz = row[nI];
  a->row_ptr = (const int*)dev;
  a->col = (const int*)(dev + b_row);
  a->val = (const z*)(dev + b_row + b_col);
  a->in_off = (const int64_t*)(dev + b_row + b_col + b_val);
  a->out_off = (const int64_t*)(dev + b_row + b_col + b_val + b_in);
  return TNT_OK;
}

int op_apply(Ctx* c, const OpApply& a) {
  int64_t total = a.B0 * a.B1 * a.B2;
  if (total <= 0) return TNT_OK;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  int nnz = a.nnz > 0 ? a.nnz : 1;
  ProfScope ps(c, "op_apply", 8.0 * (double)a.nnz * (double)total);
  k_op_apply<<<(unsigned)blocks, 256, 0, c->stream>>>(a, nnz);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

// ============================================================ vector kernels
// Deterministic reductions: a fixed grid of RB blocks; block b always covers the same
// elements in the same order; a single-block second pass sums the partials in order.
namespace {
constexpr int RB = 608;       // 4 blocks per SM (152 SMs): enough loads in flight for HBM
constexpr int RT = 256;
constexpr int KB = 8;         // vectors per multidot pass
// multidot's grid: 2 blocks per SM.  Each thread ends with 2 KV sums to reduce (five
// shuffle-adds each, on the FP64 pipe); at 4 blocks per SM a 2^20-element vector gave a
// thread only ~7 elements and the reduction rivalled the dot products themselves
constexpr int RB_DOT = 304;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of one double (result valid in thread 0)
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0;
  if (w == 0) {
    r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

// partial[v][blk] = sum over the block's range of conj(V_v[e]) w[e], v < KV; the KV
// loads of one element are independent and issued together.  The last CTA to finish (an
// arrival counter, reset by that CTA) sums the partials in block order into out[v]: the
// reduction stays deterministic and needs no second launch.
template <int KV>
__global__ void __launch_bounds__(RT) k_multidot(const z* __restrict__ V, int64_t ld,
                                                 const z* __restrict__ w, int64_t n,
                                                 z* __restrict__ partial,
                                                 const int* __restrict__ skip,
                                                 unsigned* __restrict__ counter,
                                                 z* __restrict__ out) {
  if (skip && *skip) return;  // a pass the caller decided on the device not to need
  __shared__ double sh[32];
  double ar[KV], ai[KV];
#pragma unroll
  for (int v = 0; v < KV; ++v) ar[v] = ai[v] = 0.0;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = min(n, lo + chunk);
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const z x = w[e];
    z u[KV];
#pragma unroll
    for (int v = 0; v < KV; ++v) u[v] = V[(int64_t)v * ld + e];
#pragma unroll
    for (int v = 0; v < KV; ++v) {
      ar[v] = fma(u[v].x, x.x, fma(u[v].y, x.y, ar[v]));
      ai[v] = fma(u[v].x, x.y, fma(-u[v].y, x.x, ai[v]));
    }
  }
  // all 2 KV sums in one pass: shuffles within each warp, then one barrier and a fixed-order
  // sum over the warps (the per-value block reductions cost two barriers each, and with a
  // few elements per thread they outweighed the loop)
  __shared__ double shp[RT / 32][2 * KV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < KV; ++v) {
    ar[v] = warp_sum(ar[v]);
    ai[v] = warp_sum(ai[v]);
  }
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < KV; ++v) {
      shp[wid][2 * v] = ar[v];
      shp[wid][2 * v + 1] = ai[v];
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * KV) {
    double t = 0;
#pragma unroll
    for (int q = 0; q < RT / 32; ++q) t += shp[q][threadIdx.x];
    double* po = (double*)(partial + (int64_t)(threadIdx.x >> 1) * gridDim.x + blockIdx.x);
    po[threadIdx.x & 1] = t;
    __threadfence();
  }
  // the last CTA to arrive sums every CTA's partials, in block order
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double* pp = (const double*)partial;
  double acc[2 * KV];
#pragma unroll
  for (int v = 0; v < 2 * KV; ++v) acc[v] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += RT) {
#pragma unroll
    for (int v = 0; v < KV; ++v) {
      const z pv = __ldcg(partial + (int64_t)v * gridDim.x + b);
      acc[2 * v] += pv.x;
      acc[2 * v + 1] += pv.y;
    }
  }
  (void)pp;
#pragma unroll
  for (int v = 0; v < 2 * KV; ++v) acc[v] = warp_sum(acc[v]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < 2 * KV; ++v) shp[wid][v] = acc[v];
  }
  __syncthreads();
  if (threadIdx.x < 2 * KV) {
    double t = 0;
#pragma unroll
    for (int q = 0; q < RT / 32; ++q) t += shp[q][threadIdx.x];
    ((double*)(out + (threadIdx.x >> 1)))[threadIdx.x & 1] = t;
  }
  if (threadIdx.x == 0) *counter = 0u;
  (void)sh;
}

void launch_multidot(int kv, dim3 g, dim3 b, cudaStream_t st, const z* V, int64_t ld,
                     const z* w, int64_t n, z* partial, const int* skip, unsigned* cnt,
                     z* out) {
  switch (kv) {
    case 1: k_multidot<1><<<g, b, 0, st>>>(V, ld, w, n, partial, skip, cnt, out); break;
    case 2: k_multidot<2><<<g, b, 0, st>>>(V, ld, w, n, partial, skip, cnt, out); break;
    case 3: k_multidot<3><<<g, b, 0, st>>>(V, ld, w, n, partial, skip, cnt, out); break;
    case 4: k_multidot<4><<<g, b, 0, st>>>(V, ld, w, n, partial, skip, cnt, out); break;
    case 5: k_multidot<5><<<g, b, 0, st>>>(V, ld, w, n, partial, skip, cnt, out); break;
    case 6: k_multidot<6><<<g, b, 0, st>>>(V, ld, w, n, partial, skip, cnt, out); break;
    case 7: k_multidot<7><<<g, b, 0, st>>>(V, ld, w, n, partial, skip, cnt, out); break;
    default: k_multidot<8><<<g, b, 0, st>>>(V, ld, w, n, partial, skip, cnt, out); break;
  }
}

// w[e] -= sum_v coef[v] V_v[e]; partial[blk] = sum |w[e]|^2, and the last CTA to finish
// writes the total |w|^2
__global__ void __launch_bounds__(RT) k_multiaxpy_norm(const z* __restrict__ V, int64_t ld,
                                                       int k, const z* __restrict__ coef,
                                                       z* __restrict__ w, int64_t n,
                                                       double* __restrict__ partial,
                                                       const int* __restrict__ skip,
                                                       unsigned* __restrict__ counter,
                                                       double* __restrict__ norm2_out) {
  if (skip && *skip) return;
  __shared__ z sc[64];
  __shared__ double sh[32];
  for (int t = threadIdx.x; t < k; t += blockDim.x) sc[t] = coef[t];
  __syncthreads();
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = min(n, lo + chunk);
  double acc = 0;
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    z x = w[e];
    int v = 0;
    for (; v + 8 <= k; v += 8) {  // eight independent loads in flight per thread
      z u[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) u[q] = V[(int64_t)(v + q) * ld + e];
#pragma unroll
      for (int q = 0; q < 8; ++q) {  // x -= cv u as four FMAs
        const z cv = sc[v + q];
        x.x = fma(-cv.x, u[q].x, fma(cv.y, u[q].y, x.x));
        x.y = fma(-cv.x, u[q].y, fma(-cv.y, u[q].x, x.y));
      }
    }
    for (; v < k; ++v) {
      const z u = V[(int64_t)v * ld + e];
      const z cv = sc[v];
      x.x = fma(-cv.x, u.x, fma(cv.y, u.y, x.x));
      x.y = fma(-cv.x, u.y, fma(-cv.y, u.x, x.y));
    }
    w[e] = x;
    acc = fma(x.x, x.x, fma(x.y, x.y, acc));
  }
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s;
    __threadfence();
  }
  // the last CTA to arrive sums every CTA's partial, in block order
  __shared__ bool s_last;
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double r = 0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) r += __ldcg(partial + b);
  r = block_sum(r, sh);
  if (threadIdx.x == 0) {
    *norm2_out = r;
    *counter = 0u;
  }
}

// ---------------------------------------------------------------- FP32-arithmetic passes
// The Gram-Schmidt passes of a Lanczos phase whose matvec is split TF32 (relative error
// about 2^-22): the FP64 vectors are read as they are and multiplied in FP32 with FP32
// sums per thread, warp and block; the sums over blocks, the subtraction from w and w
// itself stay FP64, so cancellation in w - V c does not amplify the FP32 rounding (the
// update's error is u_32 |V c|, like a matvec error of that size).  An SM retires 64 FP32
// FMAs per clock against 2 FP64 FMAs on GB300: these passes are bound by HBM, where the
// FP64 forms are bound by the FP64 pipe.  Conversions between the widths are integer bit
// operations on the IEEE-754 layouts (f32conv.cuh), so that no FP64-pipe instruction
// enters the element loop.
// The last CTA's sums of nv values over nb blocks (partials[v * nb + b], FP64) into
// out[v]: thread t < per nv (per the largest power of two <= RT / nv) adds blocks
// t / nv, t / nv + per, ... of value t % nv, then a fixed tree over the per copies.
// Deterministic, and a handful of FP64 adds per thread (a serial FP64 chain costs the
// FP64 pipe's full issue time per step).
__device__ void last_cta_sum(const double* __restrict__ partials, int nv, int nb,
                             double* __restrict__ out) {
  __shared__ double sp[RT];
  const int t = threadIdx.x;
  int per = 1;
  while (2 * per * nv <= RT) per *= 2;
  double r = 0;
  if (t < per * nv)
    for (int b = t / nv; b < nb; b += per) r += __ldcg(partials + (int64_t)(t % nv) * nb + b);
  sp[t] = r;
  __syncthreads();
  for (int h = per / 2; h >= 1; h >>= 1) {
    if (t < h * nv) sp[t] += sp[t + h * nv];
    __syncthreads();
  }
  if (t < nv) out[t] = sp[t];
}

template <int KV>
__global__ void __launch_bounds__(RT) k_multidot32(const z* __restrict__ V, int64_t ld,
                                                   const z* __restrict__ w, int64_t n,
                                                   double* __restrict__ partial,
                                                   unsigned* __restrict__ counter,
                                                   z* __restrict__ out) {
  float ar[KV], ai[KV];
#pragma unroll
  for (int v = 0; v < KV; ++v) ar[v] = ai[v] = 0.f;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = min(n, lo + chunk);
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const z xd = w[e];
    z u[KV];
#pragma unroll
    for (int v = 0; v < KV; ++v) u[v] = V[(int64_t)v * ld + e];
    const float xr = f32_of(xd.x), xi = f32_of(xd.y);
#pragma unroll
    for (int v = 0; v < KV; ++v) {  // conj(u) x
      const float ur = f32_of(u[v].x), ui = f32_of(u[v].y);
      ar[v] = fmaf(ur, xr, fmaf(ui, xi, ar[v]));
      ai[v] = fmaf(ur, xi, fmaf(-ui, xr, ai[v]));
    }
  }
  __shared__ float shp[RT / 32][2 * KV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < KV; ++v) {
    ar[v] = warp_sum_f(ar[v]);
    ai[v] = warp_sum_f(ai[v]);
  }
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < KV; ++v) {
      shp[wid][2 * v] = ar[v];
      shp[wid][2 * v + 1] = ai[v];
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * KV) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < RT / 32; ++q) t += shp[q][threadIdx.x];
    partial[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = f64_of(t);
    __threadfence();
  }
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  last_cta_sum(partial, 2 * KV, (int)gridDim.x, (double*)out);
  if (threadIdx.x == 0) *counter = 0u;
}

void launch_multidot32(int kv, dim3 g, dim3 b, cudaStream_t st, const z* V, int64_t ld,
                       const z* w, int64_t n, double* partial, unsigned* cnt, z* out) {
  switch (kv) {
    case 1: k_multidot32<1><<<g, b, 0, st>>>(V, ld, w, n, partial, cnt, out); break;
    case 2: k_multidot32<2><<<g, b, 0, st>>>(V, ld, w, n, partial, cnt, out); break;
    case 3: k_multidot32<3><<<g, b, 0, st>>>(V, ld, w, n, partial, cnt, out); break;
    case 4: k_multidot32<4><<<g, b, 0, st>>>(V, ld, w, n, partial, cnt, out); break;
    case 5: k_multidot32<5><<<g, b, 0, st>>>(V, ld, w, n, partial, cnt, out); break;
    case 6: k_multidot32<6><<<g, b, 0, st>>>(V, ld, w, n, partial, cnt, out); break;
    case 7: k_multidot32<7><<<g, b, 0, st>>>(V, ld, w, n, partial, cnt, out); break;
    default: k_multidot32<8><<<g, b, 0, st>>>(V, ld, w, n, partial, cnt, out); break;
  }
}

// w[e] -= sum_v coef[v] V_v[e] (the sum in FP32, the subtraction in FP64); the last CTA
// writes |w|^2 (FP32 per block, FP64 over blocks)
__global__ void __launch_bounds__(RT) k_multiaxpy_norm32(const z* __restrict__ V, int64_t ld,
                                                         int k, const z* __restrict__ coef,
                                                         z* __restrict__ w, int64_t n,
                                                         double* __restrict__ partial,
                                                         unsigned* __restrict__ counter,
                                                         double* __restrict__ norm2_out) {
  __shared__ float2 sc[64];
  __shared__ float shw[RT / 32];
  for (int t = threadIdx.x; t < k; t += blockDim.x)
    sc[t] = make_float2(f32_of(coef[t].x), f32_of(coef[t].y));
  __syncthreads();
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = min(n, lo + chunk);
  float acc = 0.f;
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    float sr = 0.f, si = 0.f;
    int v = 0;
    for (; v + 8 <= k; v += 8) {
      z u[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) u[q] = V[(int64_t)(v + q) * ld + e];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float2 cv = sc[v + q];
        const float ur = f32_of(u[q].x), ui = f32_of(u[q].y);
        sr = fmaf(cv.x, ur, fmaf(-cv.y, ui, sr));
        si = fmaf(cv.x, ui, fmaf(cv.y, ur, si));
      }
    }
    for (; v < k; ++v) {
      const z u = V[(int64_t)v * ld + e];
      const float2 cv = sc[v];
      const float ur = f32_of(u.x), ui = f32_of(u.y);
      sr = fmaf(cv.x, ur, fmaf(-cv.y, ui, sr));
      si = fmaf(cv.x, ui, fmaf(cv.y, ur, si));
    }
    z x = w[e];
    x.x -= f64_of(sr);
    x.y -= f64_of(si);
    w[e] = x;
    const float xr = f32_of(x.x), xi = f32_of(x.y);
    acc = fmaf(xr, xr, fmaf(xi, xi, acc));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  acc = warp_sum_f(acc);
  if (lane == 0) shw[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < RT / 32; ++q) t += shw[q];
    partial[blockIdx.x] = f64_of(t);
    __threadfence();
  }
  __shared__ bool s_last;
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  last_cta_sum(partial, 1, (int)gridDim.x, norm2_out);
  if (threadIdx.x == 0) *counter = 0u;
}

__global__ void k_reduce_real(const double* __restrict__ partial, int nb,
                              double* __restrict__ out, const int* __restrict__ skip) {
  if (skip && *skip) return;  // out keeps its previous value
  __shared__ double sh[32];
  double r = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) r += partial[b];
  r = block_sum(r, sh);
  if (threadIdx.x == 0) out[0] = r;
}

__global__ void k_norm2_partial(const z* __restrict__ x, int64_t n, double* __restrict__ partial) {
  __shared__ double sh[32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = min(n, lo + chunk);
  double acc = 0;
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    z v = x[e];
    acc = fma(v.x, v.x, fma(v.y, v.y, acc));
  }
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_normalize(const z* __restrict__ x, z* __restrict__ y, int64_t n,
                            const double* __restrict__ norm2) {
  // the scale by one thread of the block: an FP64 square root and division in every thread
  // cost several times the FP64-pipe issue slots of the scaling itself
  __shared__ double s_s;
  if (threadIdx.x == 0) s_s = 1.0 / sqrt(norm2[0]);
  __syncthreads();
  const double s = s_s;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = zscale(x[e], s);
}
}  // namespace

int vec_multidot(Ctx* c, const z* V, int64_t ld, int k, const z* w, int64_t n, z* d_dots,
                 const int* d_skip) {
  if (k <= 0) return TNT_OK;
  // partial sums live in scratch only until the next launch on the same stream, so the
  // region is handed back immediately (stream order serialises its reuse)
  const size_t top = c->ws.top;
  z* partial = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)KB * RB_DOT));
  c->ws.top = top;
  if (!partial) return set_err(c, TNT_E_ALLOC, "scratch exhausted (multidot)");
  for (int v0 = 0; v0 < k; v0 += KB) {
    int kv = (k - v0 < KB) ? (k - v0) : KB;
    // FP64 FLOPs (complex MAC = 8); a pass the device may skip is profiled apart, with no
    // work claimed (the host cannot know whether it ran)
    ProfScope ps(c, d_skip ? "multidot_cond" : "multidot", d_skip ? 0.0 : 8.0 * (double)kv * (double)n);
    launch_multidot(kv, RB_DOT, RT, c->stream, V + (int64_t)v0 * ld, ld, w, n, partial, d_skip,
                    c->d_count, d_dots + v0);
    c->launches += 1;
  }
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

int vec_multiaxpy_norm(Ctx* c, const z* V, int64_t ld, int k, const z* d_coef, z* w,
                       int64_t n, double* d_norm2, const int* d_skip) {
  if (k > 64) return set_err(c, TNT_E_UNSUPPORTED, "multiaxpy with k=%d > 64", k);
  const size_t top = c->ws.top;
  double* partial = (double*)ws_alloc(c, ws_round(sizeof(double) * RB));
  c->ws.top = top;
  if (!partial) return set_err(c, TNT_E_ALLOC, "scratch exhausted (multiaxpy)");
  {
    ProfScope ps(c, d_skip ? "multiaxpy_cond" : "multiaxpy",
                 d_skip ? 0.0 : (8.0 * (double)k + 4.0) * (double)n);  // FP64 FLOPs
    k_multiaxpy_norm<<<RB, RT, 0, c->stream>>>(V, ld, k, d_coef, w, n, partial, d_skip,
                                               c->d_count + 1, d_norm2);
  }
  c->launches += 1;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

int vec_multidot_f32(Ctx* c, const z* V, int64_t ld, int k, const z* w, int64_t n, z* d_dots) {
  if (k <= 0) return TNT_OK;
  const size_t top = c->ws.top;
  // four CTAs per SM: bound by HBM, these need the loads of more threads in flight than
  // the FP64 form (whose two CTAs per SM already saturate the FP64 pipe)
  double* partial = (double*)ws_alloc(c, ws_round(sizeof(double) * 2 * (size_t)KB * RB));
  c->ws.top = top;
  if (!partial) return set_err(c, TNT_E_ALLOC, "scratch exhausted (multidot32)");
  for (int v0 = 0; v0 < k; v0 += KB) {
    const int kv = (k - v0 < KB) ? (k - v0) : KB;
    ProfScope ps(c, "multidot32", 16.0 * (double)(kv + 1) * (double)n);  // bytes read
    launch_multidot32(kv, RB, RT, c->stream, V + (int64_t)v0 * ld, ld, w, n, partial,
                      c->d_count, d_dots + v0);
    c->launches += 1;
  }
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

int vec_multiaxpy_norm_f32(Ctx* c, const z* V, int64_t ld, int k, const z* d_coef, z* w,
                           int64_t n, double* d_norm2) {
  if (k > 64) return set_err(c, TNT_E_UNSUPPORTED, "multiaxpy with k=%d > 64", k);
  const size_t top = c->ws.top;
  double* partial = (double*)ws_alloc(c, ws_round(sizeof(double) * RB));
  c->ws.top = top;
  if (!partial) return set_err(c, TNT_E_ALLOC, "scratch exhausted (multiaxpy32)");
  {
    ProfScope ps(c, "multiaxpy32", 16.0 * ((double)k + 2.0) * (double)n);  // bytes moved
    k_multiaxpy_norm32<<<RB, RT, 0, c->stream>>>(V, ld, k, d_coef, w, n, partial,
                                                 c->d_count + 1, d_norm2);
  }
  c->launches += 1;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

int vec_norm2(Ctx* c, const z* x, int64_t n, double* d_norm2) {
  const size_t top = c->ws.top;
  double* partial = (double*)ws_alloc(c, ws_round(sizeof(double) * RB));
  c->ws.top = top;
  if (!partial) return set_err(c, TNT_E_ALLOC, "scratch exhausted (norm2)");
  k_norm2_partial<<<RB, RT, 0, c->stream>>>(x, n, partial);
  k_reduce_real<<<1, 256, 0, c->stream>>>(partial, RB, d_norm2, nullptr);
  c->launches += 2;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

int vec_dot(Ctx* c, const z* x, const z* y, int64_t n, z* d_dot) {
  return vec_multidot(c, x, 0, 1, y, n, d_dot);
}

int vec_normalize(Ctx* c, const z* x, z* y, int64_t n, const double* d_norm2) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > RB) blocks = RB;  // grid-stride: one scale per CTA, four CTAs per SM
  if (blocks < 1) blocks = 1;
  k_normalize<<<(unsigned)blocks, 256, 0, c->stream>>>(x, y, n, d_norm2);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

// ============================================================ tridiagonal eigensolve
// Lowest eigenpair of the Lanczos matrix T (k <= 64): multisection on the Sturm count by
// one warp (33 sub-intervals per step), then inverse iteration with a pivoted tridiagonal
// LU (thread 0).  out[0] = E, out[1] = |y_{k-1}|.
namespace {
// number of eigenvalues < x: sign changes of the leading principal minors
// p_i = (a_i - x) p_{i-1} - b_{i-1}^2 p_{i-2} (division-free Sturm sequence; a zero minor
// takes 2^-60 |p_{i-1}| with the sign opposite to its predecessor; the pair is rescaled
// by an exact power of two when its exponent leaves [-400, 400])
__device__ int sturm_count(const double* a, const double* b, int k, double x) {
  double pm2 = 1.0, pm1 = a[0] - x;
  if (pm1 == 0.0) pm1 = -0x1p-60;
  int neg_prev = __double2hiint(pm1) < 0;
  int cnt = neg_prev;
  for (int i = 1; i < k; ++i) {
    double p = fma(a[i] - x, pm1, -(b[i - 1] * b[i - 1]) * pm2);
    if (p == 0.0) p = neg_prev ? 0x1p-60 * fabs(pm1) : -0x1p-60 * fabs(pm1);
    const int neg = __double2hiint(p) < 0;
    cnt += neg != neg_prev;
    neg_prev = neg;
    pm2 = pm1;
    pm1 = p;
    const int ex = (__double2hiint(p) >> 20) & 0x7ff;
    if (ex > 1023 + 400 || ex < 1023 - 400) {
      const double f = ldexp(1.0, 1023 - ex);
      pm1 *= f;
      pm2 *= f;
    }
  }
  return cnt;
}

// one block per problem: problem p's alpha, beta, y at p * 64, out at p * 2 (skipped
// where skip[p] is set)
__global__ void k_tridiag_lowest(const double* __restrict__ alpha,
                                 const double* __restrict__ beta, int k,
                                 double* __restrict__ out, double* __restrict__ y,
                                 const int* __restrict__ skip) {
  const int pb = blockIdx.x;
  if (skip && skip[pb]) return;
  alpha += 64 * pb;
  beta += 64 * pb;
  out += 2 * pb;
  y += 64 * pb;
  __shared__ double a[64], b[64];
  __shared__ double lo_s, hi_s;
  const int l = threadIdx.x;
  for (int i = l; i < k; i += 32) a[i] = alpha[i];
  for (int i = l; i < k - 1; i += 32) b[i] = beta[i];
  __syncwarp();
  if (l == 0) {
    double lo = a[0], hi = a[0];
    for (int i = 0; i < k; ++i) {
      double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < k - 1 ? fabs(b[i]) : 0.0);
      lo = fmin(lo, a[i] - r);
      hi = fmax(hi, a[i] + r);
    }
    double pad = 1e-12 * fmax(fabs(lo), fabs(hi)) + 1e-300;
    lo_s = lo - pad;
    hi_s = hi + pad;
  }
  __syncwarp();
  double lo = lo_s, hi = hi_s;
  for (int it = 0; it < 64; ++it) {
    double width = hi - lo;
    if (width <= 4.0 * 2.220446049250313e-16 * fmax(fabs(lo), fabs(hi)) || width <= 1e-300)
      break;
    double x = lo + width * (double)(l + 1) / 33.0;
    int cnt = sturm_count(a, b, k, x);
    unsigned m = __ballot_sync(0xffffffffu, cnt >= 1);
    // smallest lane whose point lies above the lowest eigenvalue
    int first = m ? (__ffs(m) - 1) : 32;
    double nlo = lo + width * (double)first / 33.0;
    double nhi = lo + width * (double)(first + 1) / 33.0;
    if (first == 32) nhi = hi;
    lo = nlo;
    hi = nhi;
  }
  if (l == 0) {
    const double lam = 0.5 * (lo + hi);
    // inverse iteration on (T - lam I) y = y_prev with partial pivoting
    double dl[64], dm[64], du[64], du2[64], v[64];
    int piv[64];
    for (int i = 0; i < k; ++i) v[i] = 1.0 / sqrt((double)k) * (1.0 + 0.01 * i);
    const double eps = 2.220446049250313e-16;
    double scale = 0;
    for (int i = 0; i < k; ++i) scale = fmax(scale, fabs(a[i]) + (i < k - 1 ? fabs(b[i]) : 0));
    scale = fmax(scale, 1e-300);
    // T - lam I = P L U once (the shift is the same for every sweep); pivots inverted once,
    // so the three solves multiply instead of divide (a full-warp FP64 division costs
    // several FP64-pipe issue slots per lane on GB300)
    for (int i = 0; i < k; ++i) {
      dm[i] = a[i] - lam;
      du[i] = (i < k - 1) ? b[i] : 0.0;
      dl[i] = (i < k - 1) ? b[i] : 0.0;
      du2[i] = 0.0;
      piv[i] = i;
    }
    for (int i = 0; i < k - 1; ++i) {  // LU with partial pivoting (tridiagonal, textbook gtsv)
      if (fabs(dm[i]) >= fabs(dl[i])) {
        if (fabs(dm[i]) < eps * scale) dm[i] = eps * scale;
        double f = dl[i] / dm[i];
        dl[i] = f;
        dm[i + 1] -= f * du[i];
        du2[i] = 0.0;
        piv[i] = i;
      } else {
        double f = dm[i] / dl[i];
        dm[i] = dl[i];
        dl[i] = f;
        double t = du[i];
        du[i] = dm[i + 1];
        dm[i + 1] = t - f * du[i];
        if (i < k - 2) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du[i + 1];
        }
        piv[i] = i + 1;
      }
    }
    if (fabs(dm[k - 1]) < eps * scale) dm[k - 1] = eps * scale;
    for (int i = 0; i < k; ++i) dm[i] = 1.0 / dm[i];  // inverse pivots
    for (int iter = 0; iter < 3; ++iter) {
      // forward: apply row swaps and L
      for (int i = 0; i < k - 1; ++i) {
        if (piv[i] == i) {
          v[i + 1] -= dl[i] * v[i];
        } else {
          double t = v[i];
          v[i] = v[i + 1];
          v[i + 1] = t - dl[i] * v[i];
        }
      }
      // backward: U has diagonals 1/dm, du, du2; the vector is scaled down whenever an
      // entry passes 2^500 (compounding pivots of near-degenerate Ritz values)
      for (int i = k - 1; i >= 0; --i) {
        double t = v[i];
        if (i + 1 < k) t -= du[i] * v[i + 1];
        if (i + 2 < k) t -= du2[i] * v[i + 2];
        t *= dm[i];
        v[i] = t;
        if (fabs(t) > 0x1p500)
          for (int q = 0; q < k; ++q) v[q] *= 0x1p-500;
      }
      double nrm = 0;
      for (int i = 0; i < k; ++i) nrm = fma(v[i], v[i], nrm);
      const double rn = 1.0 / sqrt(nrm);
      for (int i = 0; i < k; ++i) v[i] *= rn;
    }
    // fix the sign so that the first nonzero component is positive (deterministic)
    double sgn = 1.0;
    for (int i = 0; i < k; ++i)
      if (v[i] != 0.0) {
        sgn = v[i] > 0 ? 1.0 : -1.0;
        break;
      }
    for (int i = 0; i < k; ++i) y[i] = sgn * v[i];
    out[0] = lam;
    out[1] = fabs(v[k - 1]);
  }
}
}  // namespace

int tridiag_lowest(Ctx* c, const double* d_alpha, const double* d_beta, int k, double* d_out,
                   double* d_y) {
  if (k < 1 || k > 64) return set_err(c, TNT_E_UNSUPPORTED, "tridiagonal size %d", k);
  k_tridiag_lowest<<<1, 32, 0, c->stream>>>(d_alpha, d_beta, k, d_out, d_y, nullptr);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

int tridiag_lowest_on(Ctx* c, cudaStream_t st, const double* d_alpha, const double* d_beta, int k,
                      double* d_out, double* d_y) {
  if (k < 1 || k > 64) return set_err(c, TNT_E_UNSUPPORTED, "tridiagonal size %d", k);
  k_tridiag_lowest<<<1, 32, 0, st>>>(d_alpha, d_beta, k, d_out, d_y, nullptr);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

int side_stream(Ctx* c) {
  if (c->side) return TNT_OK;
  TNT_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  for (int i = 0; i < 2; ++i) {
    TNT_CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_main[i], cudaEventDisableTiming));
    TNT_CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_side[i], cudaEventDisableTiming));
  }
  return TNT_OK;
}

int tridiag_lowest_batched(Ctx* c, const double* d_alpha, const double* d_beta, int k,
                           double* d_out, double* d_y, int nprob, const int* d_skip) {
  if (k < 1 || k > 64) return set_err(c, TNT_E_UNSUPPORTED, "tridiagonal size %d", k);
  k_tridiag_lowest<<<nprob, 32, 0, c->stream>>>(d_alpha, d_beta, k, d_out, d_y, d_skip);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

// ============================================================ gather / fill / scale
namespace {
__global__ void k_gather2d(const z* __restrict__ src, int64_t src_ld,
                           const int64_t* __restrict__ rows, int64_t nr,
                           const int64_t* __restrict__ cols, int64_t nc, z* __restrict__ dst,
                           int64_t dst_ld, int conj_t) {
  const int64_t total = nr * nc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / nc, j = e % nc;
    z v = src[rows[i] * src_ld + cols[j]];
    if (conj_t) {
      v.y = -v.y;
      dst[j * dst_ld + i] = v;
    } else {
      dst[i * dst_ld + j] = v;
    }
  }
}

__global__ void k_zfill(z* p, int64_t n, z v) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    p[e] = v;
}

// mode 0: p *= s[0]; mode 1: p *= 1/sqrt(s[0])
__global__ void k_zscale(z* p, int64_t n, const double* s, int mode) {
  __shared__ double s_f;  // by one thread, as in k_normalize
  if (threadIdx.x == 0) s_f = (mode == 0) ? s[0] : 1.0 / sqrt(s[0]);
  __syncthreads();
  const double f = s_f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    p[e] = zscale(p[e], f);
}

unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return (unsigned)b;
}
}  // namespace

int gather2d(Ctx* c, const z* src, int64_t src_ld, const int64_t* d_rows, int64_t nr,
             const int64_t* d_cols, int64_t nc, z* dst, int64_t dst_ld, int conj_t) {
  if (nr <= 0 || nc <= 0) return TNT_OK;
  k_gather2d<<<grid_for(nr * nc), 256, 0, c->stream>>>(src, src_ld, d_rows, nr, d_cols, nc,
                                                        dst, dst_ld, conj_t);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

int zfill(Ctx* c, z* p, int64_t n, z v) {
  if (n <= 0) return TNT_OK;
  k_zfill<<<grid_for(n), 256, 0, c->stream>>>(p, n, v);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

int zscale_inplace(Ctx* c, z* p, int64_t n, const double* d_scale, int mode) {
  if (n <= 0) return TNT_OK;
  k_zscale<<<grid_for(n), 256, 0, c->stream>>>(p, n, d_scale, mode);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  return TNT_OK;
}

}  // namespace tnt
