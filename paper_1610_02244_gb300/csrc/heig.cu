// Leading eigenpairs of a large Hermitian FP64 matrix (the Gram matrix of one charge block
// of the truncated SVD, App. B.1.2): k largest eigenvalues and their eigenvectors.
//
//   1. Householder reduction to real tridiagonal form G = Q T Q^H: for each column j the
//      reflector H_j = I - tau v v^H maps the part below the diagonal to beta e_1 (beta
//      real), and the trailing block is updated as A <- H_j^H A H_j through
//      p = tau A v, w = p - (tau/2)(p^H v) v, A <- A - v w^H - w v^H.
//   2. Multisection on Sturm counts of T for eigenvalues n-1, ..., n-k (one warp each),
//      to full precision.
//   3. Inverse iteration on T - lambda_i I (pivoted tridiagonal LU, three sweeps), each
//      eigenvalue its own shift; the iterates of a cluster of eigenvalues closer than
//      1e3 eps |T| are re-orthogonalised against the cluster's earlier vectors.
//   4. Back-transformation U = H_0 H_1 ... H_{n-2} Y.
//   5. Two Newton-Schulz steps U <- U (3 I - U^H U) / 2 in FP64 to restore orthonormality
//      lost to close eigenvalues.
// All arithmetic is FP64.  The cost is O(n^3) once, against O(sweeps n^3) for a Jacobi
// eigensolver.  Blocks of up to 256 rows are reduced together, one CTA each.
#include <cmath>

#include "heff_plan.cuh"

namespace tnt {

namespace {
constexpr double EPS = 2.220446049250313e-16;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// x -= a conj(b) as four FMAs (the FP64 pipe is the bottleneck of these kernels on GB300)
__device__ __forceinline__ void zsub_mul_conj(z& x, z a, z b) {
  x.x = fma(-a.x, b.x, fma(-a.y, b.y, x.x));
  x.y = fma(-a.y, b.x, fma(a.x, b.y, x.y));
}

// block-wide sum; valid in every thread on return.  The warp sums are combined by a
// butterfly over one warp's lanes (every warp the same order, so every thread gets the
// same bits): five FP64 adds per thread, where a loop over the warp sums in every thread
// cost one add per warp per thread (the FP64 pipe is the scarce unit on GB300)
__device__ double block_sum_all(double v, double* sh) {
  v = warp_sum_d(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

// block-wide maximum; valid in every thread on return
__device__ double block_max_all(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
  return r;
}

// ---------------------------------------------------------------- persistent reduction
// All columns in one cooperative launch, one grid barrier per column.  Entering column j
// every block holds the reflector (v_j, tau_j) in its workspace and p_j = tau_j T_j v_j is
// complete in global memory (T_j: the trailing block after column j-1).  Then:
//   every block: s_j = p_j^H v_j (from the per-block partials, same order everywhere),
//     w_j = p_j - (tau_j s_j / 2) v_j, the updated row j+1 of A, and from it reflector
//     j+1 (block 0 also stores it for the back-transformation);
//   each warp: for the rows it owns, T <- T - v_j w_j^H - w_j v_j^H, and in the same pass
//     the row's entry of p_{j+1} = tau_{j+1} T_{j+1} v_{j+1} and its share of s_{j+1};
//   grid barrier.
// Row g belongs to block g mod nb and, within it, to warp (g / nb) mod 16, so the rows
// left at every column stay spread over all blocks.  p and the
// partial sums are double-buffered by column parity.  The grid barrier spins on a
// generation counter with a %globaltimer limit; if any wait expires, an abort flag makes
// every block leave at its next barrier.
struct TriArgs {
  z* G;
  int64_t n;
  z* Hv;
  z* tau;
  double* d;
  double* e;
  z* p;                // 2 x n: p of even / odd columns
  z* part;             // 2 x nb partial sums of p^H v
  unsigned* bar;       // [0] arrivals, [1] generation
  int* abort_flag;
  int* status;
  z* gws;              // per-block workspace (4 n) when n exceeds the shared cache
};

__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// returns false if the CTA must stop (a wait expired here or elsewhere)
__device__ bool grid_barrier(const TriArgs& a) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = a.bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(a.bar, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      a.bar[0] = 0;
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      const uint64_t t0 = gtime();
      while (*gen == g) {
        if (*(volatile int*)a.abort_flag) { ok = 0; break; }
        if (gtime() - t0 > 2000000000ull) {
          atomicOr(a.status, 2);
          atomicExch(a.abort_flag, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (*(volatile int*)a.abort_flag) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Block-wide sum, valid in thread 0 only (warp 0 combines the warp sums).
__device__ double block_sum0(double v, double* sh) {
  v = warp_sum_d(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0;
  if (w == 0) r = warp_sum_d((l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0);
  return r;
}

// Householder reflector of a row x (the part below the diagonal of a column of a Hermitian
// matrix, conjugated): alpha = conj(x_0), xn2 = sum_{r>0} |x_r|^2.  H = I - tau v v^H with
// v = (1, conj(x_r) scale, ...) maps conj(x) to beta e_1, beta real.  Computed by one thread:
// a full-block FP64 square root and three divisions cost more FP64-pipe issue slots on
// GB300 than the vector work of a short column.
struct Refl {
  z tau, scale;
  double beta;
};
__device__ Refl refl_params(z alpha, double xn2, bool empty) {
  Refl R;
  if (empty || (xn2 == 0.0 && alpha.y == 0.0)) {
    R.tau = zmk(0, 0);
    R.beta = alpha.x;
    R.scale = zmk(0, 0);
  } else {
    const double nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2);
    R.beta = alpha.x >= 0 ? -nrm : nrm;
    R.tau = zmk((R.beta - alpha.x) / R.beta, -alpha.y / R.beta);
    const z den = zmk(alpha.x - R.beta, alpha.y);  // scale = 1 / (alpha - beta)
    const double dd = den.x * den.x + den.y * den.y;
    R.scale = zmk(den.x / dd, -den.y / dd);
  }
  return R;
}

// Reflector from x_r = conj(row[r]), r < m (row already in the workspace): v (length m,
// v[0] = 1), tau, beta with H^H x = beta e_1.  Every thread of the block returns the same
// tau and beta.
__device__ void make_reflector(const z* row, int64_t m, z* v, z* tau_out, double* beta_out,
                               double* sh) {
  __shared__ Refl s_refl;
  double acc = 0;
  for (int64_t r = 1 + threadIdx.x; r < m; r += blockDim.x) {
    const z x = row[r];
    acc = fma(x.x, x.x, fma(x.y, x.y, acc));
  }
  acc = block_sum0(acc, sh);
  if (threadIdx.x == 0) s_refl = refl_params(m > 0 ? zconj(row[0]) : zmk(0, 0), acc, m == 0);
  __syncthreads();
  const Refl R = s_refl;
  for (int64_t r = threadIdx.x; r < m; r += blockDim.x)
    v[r] = (r == 0) ? zmk(1, 0) : zmul(zconj(row[r]), R.scale);
  *tau_out = R.tau;
  *beta_out = R.beta;
  __syncthreads();
}

constexpr int TRI_THREADS = 512;
constexpr int TRI_WARPS = TRI_THREADS / 32;
constexpr int64_t TRI_CACHE = 2048;  // workspace in shared memory up to this n

__global__ void __launch_bounds__(TRI_THREADS) k_tridiag_persistent(TriArgs a) {
  extern __shared__ z sm_tri[];
  __shared__ double sh[32];
  __shared__ double shr[TRI_WARPS], shi[TRI_WARPS];
  __shared__ z s_cf;
  const int64_t n = a.n;
  const int nb = gridDim.x, b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // row g belongs to block g mod nb, warp (g / nb) mod TRI_WARPS: consecutive rows land on
  // different SMs, so every SM's FP64 units share each column's work
  const int64_t nwarps = (int64_t)nb * TRI_WARPS, own0 = (int64_t)b + (int64_t)nb * warp;
  z* ws = (n <= TRI_CACHE) ? sm_tri : a.gws + (int64_t)b * 4 * n;
  z* sv = ws;           // v_j
  z* sw = ws + n;       // w_j
  z* srow = ws + 2 * n; // updated row j+1
  z* sv2 = ws + 3 * n;  // v_{j+1}
  // reflector 0 from row 0, and p_0 = tau_0 T_0 v_0 over the owned rows
  z t;
  double beta;
  {
    const int64_t m = n - 1;
    for (int64_t c = threadIdx.x; c < m; c += blockDim.x) srow[c] = __ldcg(a.G + 1 + c);
    __syncthreads();
    make_reflector(srow, m, sv, &t, &beta, sh);
    if (b == 0) {
      for (int64_t c = threadIdx.x; c < m; c += blockDim.x) a.Hv[c] = sv[c];
      if (threadIdx.x == 0) {
        a.tau[0] = t;
        a.d[0] = __ldcg(a.G).x;
        if (m > 0) a.e[0] = beta;
      }
    }
    double pr = 0, pi = 0;
    for (int64_t g = own0; g < n; g += nwarps) {  // global row g = local row g - 1
      if (g < 1) continue;
      const z* row = a.G + g * n + 1;
      double sr = 0, si = 0;
#pragma unroll 4
      for (int64_t c = lane; c < m; c += 32) {
        const z x = __ldcg(row + c), y = sv[c];
        sr = fma(x.x, y.x, fma(-x.y, y.y, sr));
        si = fma(x.x, y.y, fma(x.y, y.x, si));
      }
      sr = warp_sum_d(sr);
      si = warp_sum_d(si);
      if (lane == 0) {
        const z pv = zmul(t, zmk(sr, si));
        a.p[g - 1] = pv;
        const z vr = sv[g - 1];
        pr += pv.x * vr.x + pv.y * vr.y;
        pi += pv.x * vr.y - pv.y * vr.x;
      }
    }
    if (lane == 0) { shr[warp] = pr; shi[warp] = pi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sa = 0, sb = 0;
      for (int q = 0; q < TRI_WARPS; ++q) { sa += shr[q]; sb += shi[q]; }
      a.part[b] = zmk(sa, sb);
    }
  }
  for (int64_t j = 0; j + 1 < n; ++j) {
    if (!grid_barrier(a)) return;
    const int64_t m = n - j - 1;          // size of T_j (local rows/cols 0..m-1 = global j+1..)
    const z* pj = a.p + (j & 1) * n;
    z* pn = a.p + ((j + 1) & 1) * n;
    const z* partj = a.part + (j & 1) * nb;
    z* partn = a.part + ((j + 1) & 1) * nb;
    if (warp == 0) {  // the nb partials, loaded by 32 lanes at once and summed by shuffles
      double sa = 0, sb = 0;
      for (int q = lane; q < nb; q += 32) {
        const z pq = __ldcg(partj + q);
        sa += pq.x;
        sb += pq.y;
      }
      sa = warp_sum_d(sa);
      sb = warp_sum_d(sb);
      if (lane == 0) {
        const z ts = zmul(t, zmk(sa, sb));
        s_cf = zmk(-0.5 * ts.x, -0.5 * ts.y);
      }
    }
    __syncthreads();
    const z cf = s_cf;
    for (int64_t c = threadIdx.x; c < m; c += blockDim.x) {
      const z pv = __ldcg(pj + c), vv = sv[c];
      sw[c] = zmk(fma(cf.x, vv.x, fma(-cf.y, vv.y, pv.x)), fma(cf.x, vv.y, fma(cf.y, vv.x, pv.y)));
    }
    __syncthreads();
    // updated row j+1 (local row 0), then reflector j+1 from its entries 1..m-1
    const z v0 = sv[0], w0 = sw[0];
    {
      const z* row = a.G + (j + 1) * n + j + 1;
      for (int64_t c = threadIdx.x; c < m; c += blockDim.x) {
        z x = __ldcg(row + c);
        zsub_mul_conj(x, v0, sw[c]);
        zsub_mul_conj(x, w0, sv[c]);
        srow[c] = x;
      }
    }
    __syncthreads();
    const int64_t m2 = m - 1;  // size of T_{j+1}
    z t2;
    make_reflector(srow + 1, m2, sv2, &t2, &beta, sh);
    if (b == 0) {
      for (int64_t c = threadIdx.x; c < m2; c += blockDim.x) a.Hv[(j + 1) * n + c] = sv2[c];
      if (threadIdx.x == 0) {
        a.tau[j + 1] = t2;
        a.d[j + 1] = srow[0].x;
        if (m2 > 0) a.e[j + 1] = beta;
      }
    }
    // owned rows r >= 1 of T_j: update, and dot with v_{j+1} for p_{j+1}
    double pr = 0, pi = 0;
    for (int64_t g = own0 + ((j + 2 > own0) ? ((j + 2 - own0 + nwarps - 1) / nwarps) * nwarps : 0);
         g < n; g += nwarps) {
      const int64_t r = g - (j + 1);  // local row in T_j
      z* row = a.G + g * n + j + 1;
      const z vr = sv[r], wr = sw[r];
      double sr = 0, si = 0;
#pragma unroll 4
      for (int64_t c = 1 + lane; c < m; c += 32) {
        z x = __ldcg(row + c);
        zsub_mul_conj(x, vr, sw[c]);
        zsub_mul_conj(x, wr, sv[c]);
        row[c] = x;
        const z q = sv2[c - 1];
        sr = fma(x.x, q.x, fma(-x.y, q.y, sr));
        si = fma(x.x, q.y, fma(x.y, q.x, si));
      }
      sr = warp_sum_d(sr);
      si = warp_sum_d(si);
      if (lane == 0) {
        const z pv = zmul(t2, zmk(sr, si));
        pn[r - 1] = pv;
        const z vv = sv2[r - 1];
        pr += pv.x * vv.x + pv.y * vv.y;
        pi += pv.x * vv.y - pv.y * vv.x;
      }
    }
    if (lane == 0) { shr[warp] = pr; shi[warp] = pi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sa = 0, sb = 0;
      for (int q = 0; q < TRI_WARPS; ++q) { sa += shr[q]; sb += shi[q]; }
      partn[b] = zmk(sa, sb);
    }
    // v_{j+1} becomes the current reflector
    for (int64_t c = threadIdx.x; c < m2; c += blockDim.x) sv[c] = sv2[c];
    t = t2;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- rows in shared memory
// The same column-by-column reduction for n <= TRI_ROWS_NMAX with each block's rows of the
// matrix (row g belongs to block g mod nb) resident in its shared memory for the whole
// reduction: the trailing update and the product with the next reflector touch shared
// memory only, and per column the global memory carries p (n entries), the per-block
// partial sums and the one row that is the source of the next reflector.
// Reflector j is v_j = (1, conj(x_c) s_j for c > j+1) with x row j of the updated matrix
// and s_j its scale; p_j = tau_j T_j v_j is formed without v_j as
// tau_j (T(g, j+1) + s_j sum_{c > j+1} T(g, c) conj(x_c)), so that the reflector's
// scalars (a block sum and one thread's square root and divisions) are computed while the
// rows are updated, and v_j is written out at the start of the next column.  Entering
// column j every block holds x (in sx, the entry j+1 zeroed), tau_j and s_j, and p_j with
// the per-block partial sums of p_j^H v_j is in global memory:
//   every block, one pass over the columns c > j with its loads issued first: v_j(c);
//     w_j(c) = p_j(c) + cf v_j(c), cf = -(tau_j / 2) p_j^H v_j; and
//     x'(c) = T_j(j+1, c) - conj(w_j(c)) - w_j(j+1) conj(v_j(c)), row j+1 after the
//     update (v_j(j+1) = 1), into sx, with the sum of |x'(c)|^2 over c > j+2;
//   each block, its rows g > j+1 of T_j, split evenly over its warps (a warp spans at most
//     two rows): T <- T - v_j w_j^H - w_j v_j^H and sum_c T(g, c) conj(x'(c)); the owner
//     of row j+2 also stores it in global memory for the next column;
//   warp 0: reflector j+1 (alpha = conj(x'(j+2))), then p_{j+1}(g) for the block's rows
//     and the block's share of p_{j+1}^H v_{j+1};
//   grid barrier.
// Vectors are indexed by global row.  Per column a block spends 16 FP64 operations per
// trailing entry on the shared vectors and 12 per entry of its rows.
constexpr int TRI_ROWS_MAX = 8;         // rows per block
static_assert(TRI_WARPS == 16, "the flattened row split divides by 16 with shifts");
constexpr int TRI_VEC = 3;              // vector entries per thread
constexpr int64_t TRI_ROWS_NMAX = 1216; // <= TRI_VEC * TRI_THREADS; (8 + 3) n entries fit

// (a, b) summed over the warp with five FP64 adds (the two sums share each step); every
// lane returns both
__device__ __forceinline__ void warp_sum_pair(double& a, double& b) {
  const bool up = (threadIdx.x & 16) != 0;
  double v = (up ? b : a) + __shfl_xor_sync(0xffffffffu, up ? a : b, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  a = __shfl_sync(0xffffffffu, v, 0);
  b = __shfl_sync(0xffffffffu, v, 16);
}

struct RowsShared {
  double br[TRI_WARPS][2], bi[TRI_WARPS][2];  // per warp, per row segment: sum T conj(x)
  double nrm[TRI_WARPS];                       // per warp: sum |x|^2
  Refl rf;                                     // reflector of the column being finished
  z cf, alpha;
};

// Rows g >= lo of this block (rows[i] = row b + nb i, R of them), flattened over
// (row, column) and split evenly over the warps: with UPD,
// T(g, c) -= v(g) conj(w(c)) + w(g) conj(v(c)) for c >= lo (the row g == lo also to
// grow); the sum over c >= lo of T(g, c) conj(x(c)) into S.br/bi[warp][segment].
template <bool UPD>
__device__ void rows_update(z* rows, int R, int b, int nb, int64_t n, int64_t lo,
                            const z* v, const z* w, const z* x, z* grow, RowsShared& S) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = (lo > b) ? (int)((lo - b + nb - 1) / nb) : 0;
  const int ract = R - i0 > 0 ? R - i0 : 0;
  // warp w covers [f0, f1) of the flattened (row, column) range, f0 = ract L w / 16, and
  // starts in row floor(ract w / 16) (exact: floor(floor(x) / L) = floor(x / L)); all in
  // 32-bit multiplies and shifts (ract L <= 8 * 1216)
  const unsigned L = (unsigned)(n - lo), total = (unsigned)ract * L;
  const unsigned f0 = (total * (unsigned)warp) >> 4, f1 = (total * (unsigned)(warp + 1)) >> 4;
  const int r0 = (ract * warp) >> 4;
#pragma unroll
  for (int seg = 0; seg < 2; ++seg) {
    double sr = 0, si = 0;
    const int ri = r0 + seg;  // row of this segment
    const int64_t s0 = (seg == 0) ? (int64_t)f0 - (int64_t)ri * L : 0;
    const int64_t s1 = min((int64_t)L, (int64_t)f1 - (int64_t)ri * L);
    if (ri < ract && s0 < s1) {
      const int i = i0 + ri;
      const int64_t g = b + (int64_t)nb * i;
      z* rw = rows + (int64_t)i * n;
      z vr = zmk(0, 0), wr = zmk(0, 0);
      if (UPD) {
        vr = v[g];
        wr = w[g];
      }
      z* gout = (UPD && g == lo) ? grow : nullptr;
#pragma unroll 2
      for (int64_t c = lo + s0 + lane; c < lo + s1; c += 32) {
        z t = rw[c];
        if (UPD) {
          zsub_mul_conj(t, vr, w[c]);
          zsub_mul_conj(t, wr, v[c]);
          rw[c] = t;
          if (gout) gout[c] = t;
        }
        const z y = x[c];  // t conj(y)
        sr = fma(t.x, y.x, fma(t.y, y.y, sr));
        si = fma(t.y, y.x, fma(-t.x, y.y, si));
      }
    }
    warp_sum_pair(sr, si);
    if (lane == 0) {
      S.br[warp][seg] = sr;
      S.bi[warp][seg] = si;
    }
  }
}

// Warp 0 after rows_update: reflector from (alpha, the block's sum of |x|^2 in S.nrm) for
// the column whose trailing block starts at lo; p(g) = tau (T(g, lo) + s sum) for the
// block's rows g >= lo into pout, the block's sum of conj(p(g)) v(g) into *partout
// (v(lo) = 1, v(c) = conj(x(c)) s).  Lane 0 returns the reflector in S.rf.
__device__ void rows_finish(const z* rows, int R, int b, int nb, int64_t n, int64_t lo,
                            const z* x, bool empty, z* pout, z* partout, RowsShared& S) {
  const int lane = threadIdx.x & 31;
  double nr = lane < TRI_WARPS ? S.nrm[lane] : 0.0;
  nr = warp_sum_d(nr);
  if (lane == 0) S.rf = refl_params(empty ? zmk(0, 0) : S.alpha, nr, empty);
  __syncwarp();
  const Refl rf = S.rf;
  const int i0 = (lo > b) ? (int)((lo - b + nb - 1) / nb) : 0;
  const int ract = R - i0 > 0 ? R - i0 : 0;
  const unsigned L = (unsigned)(n - lo), total = (unsigned)ract * L;
  double pr = 0, pi = 0;
  if (lane < ract) {
    double sr = 0, si = 0;
    for (int w = 0; w < TRI_WARPS; ++w) {  // the warps whose range meets row `lane`, in order
      const unsigned f0 = (total * (unsigned)w) >> 4, f1 = (total * (unsigned)(w + 1)) >> 4;
      const int r0 = (ract * w) >> 4;
      if (f0 < f1 && r0 == lane) {
        sr += S.br[w][0];
        si += S.bi[w][0];
      } else if (f0 < f1 && r0 + 1 == lane && f1 > (unsigned)lane * L) {
        sr += S.br[w][1];
        si += S.bi[w][1];
      }
    }
    const int64_t g = b + (int64_t)nb * (i0 + lane);
    const z t0 = rows[(int64_t)(i0 + lane) * n + lo];
    const z q = zmk(t0.x + rf.scale.x * sr - rf.scale.y * si, t0.y + rf.scale.x * si + rf.scale.y * sr);
    const z pv = zmul(rf.tau, q);
    pout[g] = pv;
    const z vg = (g == lo) ? zmk(1, 0) : zmul(zconj(x[g]), rf.scale);
    pr = pv.x * vg.x + pv.y * vg.y;
    pi = pv.x * vg.y - pv.y * vg.x;
  }
  warp_sum_pair(pr, pi);
  if (lane == 0) *partout = zmk(pr, pi);
}

__global__ void __launch_bounds__(TRI_THREADS) k_tridiag_rows(TriArgs a) {
  extern __shared__ z sm_tri[];
  __shared__ RowsShared S;
  const int64_t n = a.n;
  const int nb = gridDim.x, b = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rmax = (int)((n + nb - 1) / nb);
  const int R = (b < n) ? (int)((n - b + nb - 1) / nb) : 0;
  z* rows = sm_tri;
  z* sv = rows + (int64_t)rmax * n;  // v_j
  z* sw = sv + n;                    // w_j
  z* sx = sw + n;                    // x of the next reflector (its first entry zeroed)
  for (int i = 0; i < R; ++i) {
    const z* src = a.G + (b + (int64_t)nb * i) * n;
    for (int64_t c = tid; c < n; c += TRI_THREADS) rows[(int64_t)i * n + c] = __ldcg(src + c);
  }
  {  // reflector 0 from row 0 (columns 1..n-1), and p_0
    double acc = 0;
#pragma unroll
    for (int k = 0; k < TRI_VEC; ++k) {
      const int64_t c = 1 + tid + (int64_t)k * TRI_THREADS;
      if (c < n) {
        const z xc = __ldcg(a.G + c);
        if (c == 1) S.alpha = zconj(xc);
        else acc = fma(xc.x, xc.x, fma(xc.y, xc.y, acc));
        sx[c] = (c == 1) ? zmk(0, 0) : xc;
      }
    }
    acc = warp_sum_d(acc);
    if (lane == 0) S.nrm[warp] = acc;
    __syncthreads();
    rows_update<false>(rows, R, b, nb, n, 1, sv, sw, sx, nullptr, S);
    __syncthreads();
    if (warp == 0) {
      rows_finish(rows, R, b, nb, n, 1, sx, n < 2, a.p, a.part + b, S);
      if (b == 0 && lane == 0) {
        a.tau[0] = S.rf.tau;
        a.d[0] = __ldcg(a.G).x;
        if (n > 1) a.e[0] = S.rf.beta;
      }
    }
  }
  for (int64_t j = 0; j + 1 < n; ++j) {
    if (!grid_barrier(a)) return;
    const Refl rf = S.rf;  // reflector j
    const z* pj = a.p + (j & 1) * n;
    z* pn = a.p + ((j + 1) & 1) * n;
    const z* partj = a.part + (j & 1) * nb;
    z* partn = a.part + ((j + 1) & 1) * nb;
    const z* grow = a.G + (j + 1) * n;
    z pc[TRI_VEC], rc[TRI_VEC], vc[TRI_VEC];
#pragma unroll
    for (int k = 0; k < TRI_VEC; ++k) {
      const int64_t c = j + 1 + tid + (int64_t)k * TRI_THREADS;
      pc[k] = c < n ? __ldcg(pj + c) : zmk(0, 0);
      rc[k] = c < n ? __ldcg(grow + c) : zmk(0, 0);
    }
    const z p1 = __ldcg(pj + j + 1);
    if (warp == 0) {  // the nb partials, loaded by 32 lanes at once and summed by shuffles
      double sa = 0, sb = 0;
      for (int q = lane; q < nb; q += 32) {
        const z pq = __ldcg(partj + q);
        sa += pq.x;
        sb += pq.y;
      }
      warp_sum_pair(sa, sb);
      if (lane == 0) {
        const z ts = zmul(rf.tau, zmk(sa, sb));
        S.cf = zmk(-0.5 * ts.x, -0.5 * ts.y);
      }
    }
#pragma unroll
    for (int k = 0; k < TRI_VEC; ++k) {  // v_j, written out for the back-transformation
      const int64_t c = j + 1 + tid + (int64_t)k * TRI_THREADS;
      if (c < n) {
        vc[k] = (c == j + 1) ? zmk(1, 0) : zmul(zconj(sx[c]), rf.scale);
        sv[c] = vc[k];
        if (b == 0) a.Hv[j * n + (c - j - 1)] = vc[k];
      }
    }
    __syncthreads();
    const z cf = S.cf;
    const z w1 = zmk(p1.x + cf.x, p1.y + cf.y);  // w_j(j+1), as v_j(j+1) = 1
    double acc = 0;
    double d1 = 0;
#pragma unroll
    for (int k = 0; k < TRI_VEC; ++k) {
      const int64_t c = j + 1 + tid + (int64_t)k * TRI_THREADS;
      if (c < n) {
        const z vv = vc[k];
        const z wv = zmk(fma(cf.x, vv.x, fma(-cf.y, vv.y, pc[k].x)),
                         fma(cf.x, vv.y, fma(cf.y, vv.x, pc[k].y)));
        sw[c] = wv;
        z xn = zmk(rc[k].x - wv.x, rc[k].y + wv.y);
        zsub_mul_conj(xn, w1, vv);
        if (c == j + 1) {
          d1 = xn.x;
        } else if (c == j + 2) {
          S.alpha = zconj(xn);
          sx[c] = zmk(0, 0);
        } else {
          acc = fma(xn.x, xn.x, fma(xn.y, xn.y, acc));
          sx[c] = xn;
        }
      }
    }
    acc = warp_sum_d(acc);
    if (lane == 0) S.nrm[warp] = acc;
    __syncthreads();
    rows_update<true>(rows, R, b, nb, n, j + 2, sv, sw, sx, a.G + (j + 2) * n, S);
    __syncthreads();
    if (warp == 0) {
      const int64_t m2 = n - j - 2;  // length of reflector j+1
      rows_finish(rows, R, b, nb, n, j + 2, sx, m2 <= 0, pn, partn + b, S);
      if (b == 0 && lane == 0) {  // thread 0 holds column j+1
        a.tau[j + 1] = S.rf.tau;
        a.d[j + 1] = d1;
        if (m2 > 0) a.e[j + 1] = S.rf.beta;
      }
    }
  }
}

// ---------------------------------------------------------------- one block per CTA
// The same Householder reduction for many small Hermitian blocks (the charge blocks of a
// truncated SVD), one CTA per block and all blocks in one launch: no grid barrier, the
// block (<= TRI_CTA_MAX rows) stays in L2 and the reflector and p live in shared memory.
// On GB300 an SM retires two FP64 FMAs per clock, so a 115-row block takes about a
// millisecond on its SM while the others reduce the other blocks.  Reflector j is kept in
// row j of the block itself (columns 0..m-1), the layout the back-transformation reads:
// after column j is eliminated, row j is read no more.
constexpr int TRI_CTA_MAX = 256;
constexpr int TRI_CTA_THREADS = 256;

struct CtaBlk {
  int64_t goff;  // block (row-major, n x n) offset in the Gram buffer
  int64_t off;   // offset of its d, e, tau
  int n;
};

// Rows g >= lo of A (one warp per row): with UPD, T(g, c) -= v(g) conj(w(c)) + w(g) conj(v(c))
// for c >= lo; p(g) = tq sum_{c >= lo} T(g, c) q(c); each warp's sum of conj(p(g)) q(g) to
// s_part[.][warp].
template <bool UPD>
__device__ void cta_rows_pass(z* A, int64_t n, int64_t lo, const z* v, const z* w, const z* q,
                              z tq, z* p, double (*s_part)[TRI_CTA_THREADS / 32]) {
  constexpr int NW = TRI_CTA_THREADS / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double pr = 0, pi = 0;
  for (int64_t g = lo + warp; g < n; g += NW) {
    z* row = A + g * n;
    z vr = zmk(0, 0), wr = zmk(0, 0);
    if (UPD) {
      vr = v[g];
      wr = w[g];
    }
    double sr = 0, si = 0;
    for (int64_t c = lo + lane; c < n; c += 32) {
      z x = row[c];
      if (UPD) {
        zsub_mul_conj(x, vr, w[c]);
        zsub_mul_conj(x, wr, v[c]);
        row[c] = x;
      }
      const z y = q[c];
      sr = fma(x.x, y.x, fma(-x.y, y.y, sr));
      si = fma(x.x, y.y, fma(x.y, y.x, si));
    }
    sr = warp_sum_d(sr);
    si = warp_sum_d(si);
    if (lane == 0) {
      const z pv = zmul(tq, zmk(sr, si));
      p[g] = pv;
      const z qq = q[g];
      pr += pv.x * qq.x + pv.y * qq.y;
      pi += pv.x * qq.y - pv.y * qq.x;
    }
  }
  if (lane == 0) {
    s_part[0][warp] = pr;
    s_part[1][warp] = pi;
  }
}

// Column j: entering, v_j and p_j = tau_j T_j v_j are in shared memory with the warps'
// partial sums of p_j^H v_j.  One pass over the columns c > j gives w_j and row j+1 after
// the update (x), whose entries past j+1 give reflector j+1 (stored in row j+1 of the
// block, which is read no more); then one pass over the rows g > j+1 updates them and
// forms p_{j+1} (the trailing block is read and written once per column).  Vectors are
// indexed by row of the block; one entry per thread (n <= TRI_CTA_MAX = threads).
__global__ void __launch_bounds__(TRI_CTA_THREADS) k_tridiag_cta(z* __restrict__ G,
                                                                 const CtaBlk* __restrict__ blks,
                                                                 double* __restrict__ dAll,
                                                                 double* __restrict__ eAll,
                                                                 z* __restrict__ tauAll) {
  constexpr int NW = TRI_CTA_THREADS / 32;
  __shared__ z s_v[TRI_CTA_MAX], s_v2[TRI_CTA_MAX], s_w[TRI_CTA_MAX], s_p[TRI_CTA_MAX];
  __shared__ double sh[32];
  __shared__ double s_part[2][NW];
  __shared__ z s_cf, s_alpha;
  __shared__ Refl s_refl;
  const CtaBlk B = blks[blockIdx.x];
  const int64_t n = B.n;
  z* A = G + B.goff;
  double* d = dAll + B.off;
  double* e = eAll + B.off;
  z* tau = tauAll + B.off;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  z* v = s_v;
  z* v2 = s_v2;
  z t;
  {  // reflector 0 from row 0 (thread tid holds column 1 + tid), kept in row 0
    const int64_t c = 1 + tid;
    const z x = c < n ? A[c] : zmk(0, 0);
    double acc = (c >= 2 && c < n) ? fma(x.x, x.x, x.y * x.y) : 0.0;
    acc = block_sum0(acc, sh);
    if (tid == 0) {
      const Refl rf = refl_params(zconj(x), acc, n < 2);
      s_refl = rf;
      tau[0] = rf.tau;
      d[0] = A[0].x;
      if (n > 1) e[0] = rf.beta;
    }
    __syncthreads();
    const Refl rf = s_refl;
    t = rf.tau;
    if (c < n) {
      const z vc = (c == 1) ? zmk(1, 0) : zmul(zconj(x), rf.scale);
      v[c] = vc;
      A[c - 1] = vc;
    }
    __syncthreads();
    cta_rows_pass<false>(A, n, 1, v, s_w, v, t, s_p, s_part);
  }
  for (int64_t j = 0; j + 1 < n; ++j) {
    __syncthreads();
    const int64_t c = j + 1 + tid;
    z pc = zmk(0, 0), rc = zmk(0, 0);
    if (c < n) {
      pc = s_p[c];
      rc = A[(j + 1) * n + c];
    }
    const z p1 = s_p[j + 1];
    if (warp == 0) {
      double sa = lane < NW ? s_part[0][lane] : 0.0;
      double sb = lane < NW ? s_part[1][lane] : 0.0;
      sa = warp_sum_d(sa);
      sb = warp_sum_d(sb);
      if (lane == 0) {
        const z ts = zmul(t, zmk(sa, sb));
        s_cf = zmk(-0.5 * ts.x, -0.5 * ts.y);
      }
    }
    __syncthreads();
    const z cf = s_cf;
    const z w1 = zmk(p1.x + cf.x, p1.y + cf.y);  // w_j(j+1), as v_j(j+1) = 1
    z x = zmk(0, 0);
    double acc = 0;
    if (c < n) {
      const z vv = v[c];
      const z wv = zmk(fma(cf.x, vv.x, fma(-cf.y, vv.y, pc.x)), fma(cf.x, vv.y, fma(cf.y, vv.x, pc.y)));
      s_w[c] = wv;
      x = zmk(rc.x - wv.x, rc.y + wv.y);
      zsub_mul_conj(x, w1, vv);
      if (c >= j + 3) acc = fma(x.x, x.x, x.y * x.y);
      if (c == j + 2) s_alpha = zconj(x);
    }
    acc = block_sum0(acc, sh);
    const int64_t m2 = n - j - 2;
    if (tid == 0) {  // thread 0 holds column j+1
      const Refl rf = refl_params(m2 > 0 ? s_alpha : zmk(0, 0), acc, m2 <= 0);
      s_refl = rf;
      tau[j + 1] = rf.tau;
      d[j + 1] = x.x;
      if (m2 > 0) e[j + 1] = rf.beta;
    }
    __syncthreads();
    const Refl rf = s_refl;
    if (c >= j + 2 && c < n) {
      const z vc = (c == j + 2) ? zmk(1, 0) : zmul(zconj(x), rf.scale);
      v2[c] = vc;
      A[(j + 1) * n + (c - j - 2)] = vc;
    }
    __syncthreads();
    cta_rows_pass<true>(A, n, j + 2, v, s_w, v2, rf.tau, s_p, s_part);
    z* tmp = v;
    v = v2;
    v2 = tmp;
    t = rf.tau;
  }
}

// Number of eigenvalues of T below x from the signs of the leading principal minors
// p_i = det(T_i - x I), p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (Sturm sequence of the
// characteristic polynomials, Givens' bisection): a sign change between p_{i-1} and p_i
// marks an eigenvalue below x.  Each step is one subtraction and two products; rounding in
// a step perturbs only d_i and e_{i-1} by O(eps) relative, so the count is that of a
// matrix within O(eps |T|).  Division-free: a full-warp FP64 division costs several times
// the FP64-pipe issue slots of these three operations.  The pair (p_{i-1}, p_i) is
// rescaled by an exact power of two when its exponent leaves [-400, 400]; signs and
// exponents are read as integers.  A zero minor is replaced by 2^-60 |p_{i-1}| with the
// sign opposite to its predecessor (the tiny negative pivot of the ratio form).
__device__ __forceinline__ int hi_exp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }
__device__ int sturm_lt(const double* d, const double* e, int64_t n, double x, double pivmin) {
  (void)pivmin;
  double pm2 = 1.0, pm1 = d[0] - x;
  int neg_prev = 0;  // sign of p_0 = 1
  int cnt = 0;
  if (pm1 == 0.0) pm1 = -0x1p-60;
  int neg = __double2hiint(pm1) < 0;
  cnt += neg != neg_prev;
  neg_prev = neg;
  for (int64_t i = 1; i < n; ++i) {
    const double ei = e[i - 1];
    double p = fma(d[i] - x, pm1, -(ei * ei) * pm2);
    if (p == 0.0) p = neg_prev ? 0x1p-60 * fabs(pm1) : -0x1p-60 * fabs(pm1);
    neg = __double2hiint(p) < 0;
    cnt += neg != neg_prev;
    neg_prev = neg;
    pm2 = pm1;
    pm1 = p;
    const int ex = hi_exp(p);
    if (ex > 1023 + 400 || ex < 1023 - 400) {  // keep the pair in range: exact scaling
      const double f = ldexp(1.0, 1023 - ex);
      pm1 *= f;
      pm2 *= f;
    }
  }
  return cnt;
}

// One eigenproblem of the eigen phase, several of which share each launch (the charge
// blocks of one truncated SVD): the tridiagonal T (d, e, tau at off; n entries), its
// reflectors (row j = v_j of Hv at hoff, row stride n), and the k wanted eigenpairs, whose
// eigenvalues sit at ev[evo ..], iterates at Y[yo ..] (n k), first eigenvectors at
// U0[yo ..] (n x k, leading dimension k), inverse-iteration factors at gwork[wo ..] (6 n k).
struct EBlk {
  int64_t n, k;
  int64_t off, hoff, evo, yo, wo;
};

// Split of T at a negligible trailing block (the deflation LAPACK's tridiagonal solvers
// apply at negligible off-diagonals): the longest trailing range [s, n) whose diagonal and
// off-diagonal entries, its coupling e_{s-1} included, are all at most SPLIT_TOL |T|.  A
// rank-deficient Gram block reduces to such a T: once the reflectors have spanned the
// block's range, the trailing matrix is rounding noise (a few eps |T| and more where the
// Gram matrix itself carries the rounding of a long sum); 1e3 eps |T| catches it.  The
// split also absorbs real eigenvalues below that level (singular values under ~5e-7
// sigma_max): the canonical vectors span their subspace exactly, and the truncated SVD
// resolves its singular values in a second pass over that subspace.  The eigenvalues of that range are
// zero to within SPLIT_TOL |T|, and any orthonormal basis of its coordinates is an
// eigenbasis to that accuracy: the canonical vectors e_s, ..., e_{n-1} are taken, exactly
// orthonormal to each other and (zero beyond s) to the iterates of T[0, s), with no
// inverse iteration.  One warp per problem: |T| (Gershgorin) to tnorm, s to nr.
constexpr double SPLIT_TOL = 1e3 * 2.220446049250313e-16;
__global__ void k_split(const double* __restrict__ dAll, const double* __restrict__ eAll,
                        const EBlk* __restrict__ blks, double* __restrict__ tnorm,
                        int64_t* __restrict__ nr) {
  const int lane = threadIdx.x & 31;
  const EBlk B = blks[blockIdx.x];
  const int64_t n = B.n;
  const double* d = dAll + B.off;
  const double* e = eAll + B.off;
  double tn = 0;
  for (int64_t r = lane; r < n; r += 32)
    tn = fmax(tn, fabs(d[r]) + (r > 0 ? fabs(e[r - 1]) : 0.0) + (r < n - 1 ? fabs(e[r]) : 0.0));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
  if (lane == 0) {
    const double tol = SPLIT_TOL * tn;
    int64_t s = n;
    while (s > 0 && fabs(d[s - 1]) <= tol && (s - 1 == 0 || fabs(e[s - 2]) <= tol)) --s;
    tnorm[blockIdx.x] = tn;
    nr[blockIdx.x] = s;
  }
}

// eigenvalue of ascending index n-1-i for i < k; ev[i] descending.  One warp per
// eigenvalue: the 32 lanes evaluate Sturm counts at 32 interior points, shrinking the
// bracket 33-fold per step, to full precision (about 11 steps).  The values serve only as
// shifts (singular values are taken later as FP64 projection norms), and each SM's few
// FP64 units favour short dependent chains over many of them.  Warp g works on eigenvalue
// eig[g].y of problem eig[g].x, on the leading block T[0, s) of the split; indices from s
// on belong to the negligible block and take its diagonal entry.
__global__ void k_bisect(const double* __restrict__ dAll, const double* __restrict__ eAll,
                         const EBlk* __restrict__ blks, const int2* __restrict__ eig,
                         const int64_t* __restrict__ nrAll, const double* __restrict__ tnorm,
                         double* __restrict__ evAll) {
  const int lane = threadIdx.x & 31;
  const int2 gi = eig[blockIdx.x];
  const EBlk B = blks[gi.x];
  const int64_t n = nrAll[gi.x], i = gi.y;
  const double* d = dAll + B.off;
  const double* e = eAll + B.off;
  if (i >= n) {
    if (lane == 0) evAll[B.evo + i] = d[i];
    return;
  }
  double lo = INFINITY, hi = -INFINITY, emax2 = 0;
  for (int64_t r = lane; r < n; r += 32) {
    const double rad = (r > 0 ? fabs(e[r - 1]) : 0.0) + (r < n - 1 ? fabs(e[r]) : 0.0);
    lo = fmin(lo, d[r] - rad);
    hi = fmax(hi, d[r] + rad);
    if (r < n - 1) emax2 = fmax(emax2, e[r] * e[r]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    emax2 = fmax(emax2, __shfl_xor_sync(0xffffffffu, emax2, o));
  }
  const double tn = tnorm[gi.x];
  const double pivmin = fmax(1e-300, EPS * EPS * fmax(emax2, 1e-300)) + 1e-300;
  const int64_t idx = n - 1 - i;
  const double pad = 2 * EPS * tn + 1e-300;
  lo -= pad;
  hi += pad;
  const double tol = 1e-300;  // full precision: the shifts must resolve close eigenvalues
  for (int it = 0; it < 64; ++it) {
    const double width = hi - lo;
    if (width <= fmax(tol, 4 * EPS * fmax(fabs(lo), fabs(hi)))) break;
    const double x = lo + width * (double)(lane + 1) / 33.0;
    const unsigned below = __ballot_sync(0xffffffffu, sturm_lt(d, e, n, x, pivmin) <= idx);
    const int p = __popc(below);  // points left of eigenvalue idx (counts are monotone)
    const double nlo = p > 0 ? lo + width * (double)p / 33.0 : lo;
    const double nhi = p < 32 ? lo + width * (double)(p + 1) / 33.0 : hi;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) evAll[B.evo + i] = 0.5 * (lo + hi);
}

// Inverse iteration on T - lambda_i I, one shift per eigenvalue.  Eigenvalues whose
// consecutive gaps are below IV_ORTOL |T| = 1e3 eps |T| form a cluster (in a truncated
// SVD's Gram block, typically the rounding-level eigenvalues of a rank-deficient block),
// handled by one CTA: each member's thread factors T - lambda_i I with its
// own eigenvalue as the shift (pivoted tridiagonal LU in the member's slice of gwork), every
// sweep solves all members at once (one thread per member, the recurrences are serial) and
// re-orthogonalises the members in order (classical Gram-Schmidt, twice, then a max-scaled
// normalisation), so coincident eigenvalues still give independent vectors.  With its own
// shift a member's iterate is dominated by its own eigenvector after each solve; a shared
// shift (the cluster head's) left the members far from it dominated by the eigenvector
// just outside the cluster, nearly parallel to that vector's own iterate, and Newton-Schulz
// cannot restore a basis that far from orthonormal.  Outside a cluster an iterate is
// accurate to about eps |T| / gap <= eps / IV_ORTOL, which the final Newton-Schulz steps
// absorb.  The iterates are the output columns Y[i * n ...] themselves.
constexpr int IV_THREADS = 128;
constexpr int IV_CHUNK = 1024;   // earlier cluster members handled per Gram-Schmidt chunk
constexpr double IV_ORTOL = 1e3 * 2.220446049250313e-16;

// LU with partial pivoting of T - lam I (tridiagonal, textbook); factors in w[0 .. 5n):
// dl, dm, du, du2 (n each), then n pivot bytes.  Pivots are floored at +-small in both
// branches so that the solve never divides by less than eps |T|.
__device__ void iv_factor(const double* d, const double* e, int64_t n, double lam, double small,
                          double* w) {
  double* dl = w;
  double* dm = w + n;
  double* du = w + 2 * n;
  double* du2 = w + 3 * n;
  int8_t* piv = (int8_t*)(w + 4 * n);
  for (int64_t r = 0; r < n; ++r) {
    dm[r] = d[r] - lam;
    du[r] = r < n - 1 ? e[r] : 0.0;
    dl[r] = r < n - 1 ? e[r] : 0.0;
    du2[r] = 0.0;
  }
  for (int64_t r = 0; r < n - 1; ++r) {
    const double a = dm[r], b = dl[r];
    if (fabs(a) >= fabs(b)) {
      const double aa = fabs(a) < small ? (a < 0 ? -small : small) : a;
      dm[r] = aa;
      const double f = b / aa;
      dl[r] = f;
      dm[r + 1] -= f * du[r];
      piv[r] = 0;
    } else {
      const double bb = fabs(b) < small ? (b < 0 ? -small : small) : b;
      const double f = a / bb;
      dm[r] = bb;
      dl[r] = f;
      const double t = du[r];
      du[r] = dm[r + 1];
      dm[r + 1] = t - f * du[r];
      if (r < n - 2) {
        du2[r] = du[r + 1];
        du[r + 1] = -f * du[r + 1];
      }
      piv[r] = 1;
    }
  }
  if (fabs(dm[n - 1]) < small) dm[n - 1] = dm[n - 1] < 0 ? -small : small;
}

// solve (T - lambda I) y = y in place from the factors of iv_factor; the vector is scaled
// down whenever an entry passes 2^500 (compounding pivots of near-degenerate eigenvalues:
// the solution of a scaled system is the scaled solution)
__device__ void iv_solve(double* y, int64_t n, const double* w) {
  const double* dl = w;
  const double* dm = w + n;
  const double* du = w + 2 * n;
  const double* du2 = w + 3 * n;
  const int8_t* piv = (const int8_t*)(w + 4 * n);
  for (int64_t r = 0; r < n - 1; ++r) {
    if (piv[r] == 0) {
      y[r + 1] -= dl[r] * y[r];
    } else {
      const double t = y[r];
      y[r] = y[r + 1];
      y[r + 1] = t - dl[r] * y[r];
    }
  }
  for (int64_t r = n - 1; r >= 0; --r) {
    double v = y[r];
    if (r + 1 < n) v -= du[r] * y[r + 1];
    if (r + 2 < n) v -= du2[r] * y[r + 2];
    v /= dm[r];
    y[r] = v;
    if (fabs(v) > 0x1p500)
      for (int64_t q = 0; q < n; ++q) y[q] *= 0x1p-500;
  }
}

__global__ void __launch_bounds__(IV_THREADS) k_inviter(
    const double* __restrict__ dAll, const double* __restrict__ eAll,
    const EBlk* __restrict__ blks, const int2* __restrict__ eig,
    const int64_t* __restrict__ nrAll, const double* __restrict__ evAll,
    const double* __restrict__ tnorm, double* __restrict__ gworkAll, double* __restrict__ YAll) {
  __shared__ double sdot[IV_CHUNK];
  __shared__ double sh[32];
  const int2 gi = eig[blockIdx.x];
  const EBlk B = blks[gi.x];
  const int64_t nfull = B.n, i0 = gi.y;
  const int64_t n = nrAll[gi.x];          // the leading block of the split
  const int64_t k = min(B.k, n);          // eigenpairs of the leading block
  const double* d = dAll + B.off;
  const double* e = eAll + B.off;
  const double* ev = evAll + B.evo;
  double* gwork = gworkAll + B.wo;
  double* Y = YAll + B.yo;
  if (i0 >= n) {  // an index of the negligible trailing block: the canonical vector e_i0
    for (int64_t r = threadIdx.x; r < nfull; r += blockDim.x) Y[i0 * nfull + r] = (r == i0) ? 1.0 : 0.0;
    return;
  }
  // |T| floored well inside the normal range: a zero block (a charge sector of theta with
  // no weight) has T = 0, and pivots of eps |T| would then be denormal and the solves
  // would overflow; with the floor its eigenvectors come out as orthonormal start vectors
  const double tn = fmax(tnorm[gi.x], 1e-200);
  const double ortol = IV_ORTOL * tn;
  if (i0 > 0 && ev[i0 - 1] - ev[i0] < ortol) return;  // not the head of its cluster
  int64_t i1 = i0 + 1;
  while (i1 < k && ev[i1 - 1] - ev[i1] < ortol) ++i1;
  const double small = EPS * tn;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nwarps = IV_THREADS / 32;
  // each member's own factorisation, in its own 6n-double slice of gwork
  for (int64_t i = i0 + tid; i < i1; i += IV_THREADS) iv_factor(d, e, n, ev[i], small, gwork + i * (6 * n));
  // deterministic start vectors, free of structure, distinct per member
  for (int64_t i = i0; i < i1; ++i)
    for (int64_t r = tid; r < nfull; r += IV_THREADS) {
      uint32_t h = 2166136261u ^ (uint32_t)(i * 2654435761u) ^ (uint32_t)(r * 2246822519u);
      h *= 16777619u;
      h ^= h >> 15;
      h *= 2654435761u;
      Y[i * nfull + r] = r < n ? 0.5 + (double)(h & 0xffff) / 65536.0 : 0.0;
    }
  __syncthreads();
  for (int sweep = 0; sweep < 3; ++sweep) {
    for (int64_t i = i0 + tid; i < i1; i += IV_THREADS) iv_solve(Y + i * nfull, n, gwork + i * (6 * n));
    __syncthreads();
    for (int64_t i = i0; i < i1; ++i) {
      double* y = Y + i * nfull;
      for (int pass = 0; pass < 2 && i > i0; ++pass) {
        for (int64_t q0 = i0; q0 < i; q0 += IV_CHUNK) {
          const int64_t q1 = min(i, q0 + IV_CHUNK);
          for (int64_t q = q0 + warp; q < q1; q += nwarps) {  // one warp per dot product
            const double* yq = Y + q * nfull;
            double acc = 0;
            for (int64_t r = lane; r < n; r += 32) acc = fma(y[r], yq[r], acc);
            acc = warp_sum_d(acc);
            if (lane == 0) sdot[q - q0] = acc;
          }
          __syncthreads();
          for (int64_t r = tid; r < n; r += IV_THREADS) {
            double v = y[r];
            for (int64_t q = q0; q < q1; ++q) v = fma(-sdot[q - q0], Y[q * nfull + r], v);
            y[r] = v;
          }
          __syncthreads();
        }
      }
      // norm of y / max|y|: the solve can return entries near 1 / (eps |T|), whose squares
      // would overflow
      double mx = 0;
      for (int64_t r = tid; r < n; r += IV_THREADS) mx = fmax(mx, fabs(y[r]));
      mx = block_max_all(mx, sh);
      const double sc = mx > 0 ? 1.0 / mx : 0.0;
      double acc = 0;
      for (int64_t r = tid; r < n; r += IV_THREADS) {
        const double v = y[r] * sc;
        acc = fma(v, v, acc);
      }
      acc = block_sum_all(acc, sh);
      const double inv = acc > 0 ? sc / sqrt(acc) : 0.0;
      for (int64_t r = tid; r < n; r += IV_THREADS) y[r] *= inv;
      __syncthreads();
    }
  }
}

// U[:, i] = H_0 ... H_{n-2} y_i; one CTA per BT_COLS eigenvectors of one problem
// (bt[g] = (problem, first column)), held in shared memory.  Each reflector is read once
// per CTA for all its columns, and the CTA's reduction of the BT_COLS dot products is one
// pass: the FP64 pipe, not the reflector loads or the synchronisation, sets the pace.
constexpr int BT_COLS = 2;
__global__ void __launch_bounds__(256) k_backtransform(const double* __restrict__ YAll,
                                                       const z* __restrict__ HvAll,
                                                       const z* __restrict__ tauAll,
                                                       const EBlk* __restrict__ blks,
                                                       const int2* __restrict__ bt, int cols,
                                                       z* __restrict__ U0All) {
  extern __shared__ double sm_bt[];
  z* y = (z*)sm_bt;  // cols x n (cols = BT_COLS, or 1 when two vectors do not fit)
  __shared__ double shr[8][BT_COLS], shi[8][BT_COLS];
  __shared__ z s_ts[BT_COLS];
  const int2 gb = bt[blockIdx.x];
  const EBlk B = blks[gb.x];
  const int64_t n = B.n, k = B.k, i0 = gb.y;
  const double* Y = YAll + B.yo;
  const z* Hv = HvAll + B.hoff;
  const z* tau = tauAll + B.off;
  z* U = U0All + B.yo;  // n x k, leading dimension k
  const int ncol = (k - i0 < cols) ? (int)(k - i0) : cols;
  for (int q = 0; q < cols; ++q)
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x)
      y[q * n + r] = zmk(q < ncol ? Y[(i0 + q) * n + r] : 0.0, 0);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t j = n - 2; j >= 0; --j) {
    const z t = tau[j];
    if (t.x == 0.0 && t.y == 0.0) continue;
    const int64_t m = n - j - 1;
    const z* v = Hv + j * n;
    double sr[BT_COLS], si[BT_COLS];  // s = v^H y[j+1:] per column
#pragma unroll
    for (int q = 0; q < BT_COLS; ++q) sr[q] = si[q] = 0;
    for (int64_t r = threadIdx.x; r < m; r += blockDim.x) {
      const z a = v[r];
#pragma unroll
      for (int q = 0; q < BT_COLS; ++q) {
        if (q >= cols) break;
        const z b = y[q * n + j + 1 + r];
        sr[q] = fma(a.x, b.x, fma(a.y, b.y, sr[q]));
        si[q] = fma(a.x, b.y, fma(-a.y, b.x, si[q]));
      }
    }
#pragma unroll
    for (int q = 0; q < BT_COLS; ++q) {
      sr[q] = warp_sum_d(sr[q]);
      si[q] = warp_sum_d(si[q]);
      if (lane == 0) {
        shr[warp][q] = sr[q];
        shi[warp][q] = si[q];
      }
    }
    __syncthreads();
    if (threadIdx.x < cols) {
      double a = 0, b = 0;
      for (int w = 0; w < 8; ++w) {
        a += shr[w][threadIdx.x];
        b += shi[w][threadIdx.x];
      }
      s_ts[threadIdx.x] = zmul(t, zmk(a, b));
    }
    __syncthreads();
    for (int64_t r = threadIdx.x; r < m; r += blockDim.x) {
      const z a = v[r];
#pragma unroll
      for (int q = 0; q < BT_COLS; ++q) {
        if (q >= cols) break;
        z* p = y + q * n + j + 1 + r;
        const z ts = s_ts[q];
        z x = *p;
        x.x = fma(-ts.x, a.x, fma(ts.y, a.y, x.x));
        x.y = fma(-ts.x, a.y, fma(-ts.y, a.x, x.y));
        *p = x;
      }
    }
    __syncthreads();
  }
  for (int q = 0; q < ncol; ++q)
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) U[r * k + i0 + q] = y[q * n + r];
}

// Small complex GEMMs of many problems in one launch (the Newton-Schulz steps of the
// eigen phase): task t computes C = op(A) B, op(A)(i, l) = A[i a_rs + l a_cs] (conjugated
// if conj_a), B(l, j) = B[l b_rs + j b_cs], C(i, j) = C[i c_rs + j]; one 16 x 16 output
// tile per CTA iteration, tiles[g] = (task, m0, n0).  coef != 0 instead writes
// C = 1.5 I - 0.5 op(A) B (the Newton-Schulz coefficient matrix).
struct NsTask {
  int64_t M, N, K;
  const z* A;
  int64_t a_rs, a_cs;
  const z* B;
  int64_t b_rs, b_cs;
  z* C;
  int64_t c_rs;
  int conj_a, coef;
};
__global__ void __launch_bounds__(256) k_gemm_tasks(const NsTask* __restrict__ tasks,
                                                    const int4* __restrict__ tiles, int ntiles) {
  __shared__ z As[16][17];
  __shared__ z Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int4 tl = tiles[t];
    const NsTask tk = tasks[tl.x];
    z acc = zmk(0, 0);
    for (int64_t k0 = 0; k0 < tk.K; k0 += 16) {
      {
        const int64_t gi = tl.y + ty, gk = k0 + tx;
        z v = (gi < tk.M && gk < tk.K) ? tk.A[gi * tk.a_rs + gk * tk.a_cs] : zmk(0, 0);
        if (tk.conj_a) v.y = -v.y;
        As[ty][tx] = v;
      }
      {
        const int64_t gk = k0 + ty, gj = tl.z + tx;
        Bs[ty][tx] = (gj < tk.N && gk < tk.K) ? tk.B[gk * tk.b_rs + gj * tk.b_cs] : zmk(0, 0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) zfma(acc, As[ty][kk], Bs[kk][tx]);
      __syncthreads();
    }
    const int64_t gi = tl.y + ty, gj = tl.z + tx;
    if (gi < tk.M && gj < tk.N) {
      if (tk.coef) {
        acc = zscale(acc, -0.5);
        if (gi == gj) acc.x += 1.5;
      }
      tk.C[gi * tk.c_rs + gj] = acc;
    }
  }
}

// S <- 1.5 I - 0.5 S  (k x k)
__global__ void k_ns_coef(z* S, int64_t k) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < k * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k, c = e % k;
    z v = zscale(S[e], -0.5);
    if (r == c) v.x += 1.5;
    S[e] = v;
  }
}

__global__ void k_copy_cols(const z* __restrict__ src, int64_t n, int64_t k, int64_t lds,
                            z* __restrict__ dst, int64_t ldd) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k, c = e % k;
    dst[r * ldd + c] = src[r * lds + c];
  }
}

unsigned gsz(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return (unsigned)b;
}
}  // namespace

constexpr int TRI_MAX_BLOCKS = 1216;

size_t heig_scratch_bound(int64_t n, int64_t k) {
  const size_t gws = n > TRI_CACHE ? ws_round(sizeof(z) * 4 * n * TRI_MAX_BLOCKS) : 0;
  return ws_round(sizeof(z) * n * n) + 3 * ws_round(sizeof(z) * n) + 3 * ws_round(sizeof(double) * n) +
         gws + ws_round(sizeof(z) * 2 * TRI_MAX_BLOCKS) + ws_round(sizeof(double) * k) +
         ws_round(sizeof(double) * (6 * n * k + k)) +
         ws_round(sizeof(double) * n * k) + 2 * ws_round(sizeof(z) * n * k) + 2 * ws_round(sizeof(z) * k * k) +
         (size_t)(1 << 20);
}

// Second half of the eigensolve: from the tridiagonal form (d, e) and its reflectors
// (Hv, row j = v_j, row stride n; tau) to the eigenvectors of the k largest eigenvalues
// in U (n x k, leading dimension ldu), descending; ev (device, k).
int heig_finish(Ctx* c, int64_t n, int64_t k, const z* Hv, const z* tau, const double* d,
                const double* e, z* U, int64_t ldu, double* ev) {
  const size_t top = c->ws.top;
  double* tn = (double*)ws_alloc(c, ws_round(sizeof(double)));
  int64_t* nr = (int64_t*)ws_alloc(c, ws_round(sizeof(int64_t)));
  double* work = (double*)ws_alloc(c, ws_round(sizeof(double) * (6 * n * k + k)));
  double* Y = (double*)ws_alloc(c, ws_round(sizeof(double) * n * k));
  z* U0 = (z*)ws_alloc(c, ws_round(sizeof(z) * n * k));
  z* S = (z*)ws_alloc(c, ws_round(sizeof(z) * k * k));
  EBlk* dblk = (EBlk*)ws_alloc(c, ws_round(sizeof(EBlk)));
  int2* deig = (int2*)ws_alloc(c, ws_round(sizeof(int2) * (size_t)(2 * k + 2)));
  if (!tn || !nr || !work || !Y || !U0 || !S || !dblk || !deig) {
    c->ws.top = top;
    return set_err(c, TNT_E_ALLOC, "scratch exhausted (eigenvectors n=%lld k=%lld)", (long long)n, (long long)k);
  }
  cudaStream_t st = c->stream;
  const int cols = (sizeof(z) * n * BT_COLS <= (size_t)200 * 1024) ? BT_COLS : 1;
  const int64_t nbt = (k + cols - 1) / cols;
  {  // one problem: the block table and the (eigenvalue, back-transformation) index tables
    const EBlk hb{n, k, 0, 0, 0, 0, 0};
    std::vector<int2> he((size_t)(k + nbt));
    for (int64_t i = 0; i < k; ++i) he[(size_t)i] = make_int2(0, (int)i);
    for (int64_t q = 0; q < nbt; ++q) he[(size_t)(k + q)] = make_int2(0, (int)(q * cols));
    TNT_CUDA_TRY(c, cudaMemcpyAsync(dblk, &hb, sizeof(EBlk), cudaMemcpyHostToDevice, st));
    TNT_CUDA_TRY(c, cudaMemcpyAsync(deig, he.data(), sizeof(int2) * he.size(), cudaMemcpyHostToDevice, st));
    TNT_CUDA_TRY(c, cudaStreamSynchronize(st));  // the host tables die at the end of scope
  }
  {
    ProfScope ps(c, "heig_tridiag_eig");
    k_split<<<1, 32, 0, st>>>(d, e, dblk, tn, nr);
    k_bisect<<<(unsigned)k, 32, 0, st>>>(d, e, dblk, deig, nr, tn, ev);
    k_inviter<<<(unsigned)k, IV_THREADS, 0, st>>>(d, e, dblk, deig, nr, ev, tn, work, Y);
    c->launches += 2;
    TNT_CHECK_LAUNCH(c);
  }
  {
    ProfScope ps(c, "heig_backtransform", 8.0 * (double)n * (double)n * (double)k);
    const size_t smem = sizeof(z) * n * cols;
    TNT_CUDA_TRY(c, cudaFuncSetAttribute(k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_backtransform<<<(unsigned)nbt, 256, smem, st>>>(Y, Hv, tau, dblk, deig + k, cols, U0);
    c->launches++;
    TNT_CHECK_LAUNCH(c);
  }
  // two Newton-Schulz steps: S = X^H X; S <- 1.5 I - 0.5 S; X <- X S  (U0 -> U -> U0 -> U)
  int r = TNT_OK;
  z* src = U0;
  int64_t lds = k;
  for (int step = 0; step < 2 && r == TNT_OK; ++step) {
    z* dst = (step == 0) ? U : U0;
    const int64_t ldd = (step == 0) ? ldu : k;
    ZGemm g{};
    g.M = k; g.N = k; g.K = n;
    g.A = src; g.a_rs = 1; g.a_cs = lds; g.conj_a = 1;
    g.B = src; g.b_rs = lds; g.b_cs = 1;
    g.C = S; g.c_rs = k;
    g.alpha = zmk(1, 0); g.beta = zmk(0, 0); g.batch = 1;
    r = zgemm(c, g);
    if (r != TNT_OK) break;
    k_ns_coef<<<gsz(k * k), 256, 0, st>>>(S, k);
    c->launches++;
    ZGemm h{};
    h.M = n; h.N = k; h.K = k;
    h.A = src; h.a_rs = lds; h.a_cs = 1;
    h.B = S; h.b_rs = k; h.b_cs = 1;
    h.C = dst; h.c_rs = ldd;
    h.alpha = zmk(1, 0); h.beta = zmk(0, 0); h.batch = 1;
    r = zgemm(c, h);
    src = dst;
    lds = ldd;
  }
  if (r == TNT_OK) {
    k_copy_cols<<<gsz(n * k), 256, 0, st>>>(U0, n, k, k, U, ldu);
    c->launches++;
  }
  c->ws.top = top;
  return r;
}

// G (n x n, row-major, Hermitian, destroyed); U (n x k, leading dimension ldu): the
// eigenvectors of the k largest eigenvalues, in descending order; ev (device, k).
int heig_top(Ctx* c, z* G, int64_t n, int64_t k, z* U, int64_t ldu, double* ev) {
  if (k < 1 || k > n) return set_err(c, TNT_E_INVALID, "heig_top: k = %lld of n = %lld", (long long)k, (long long)n);
  if (n > 8192) return set_err(c, TNT_E_UNSUPPORTED, "heig_top: n = %lld > 8192", (long long)n);
  const size_t top = c->ws.top;
  z* Hv = (z*)ws_alloc(c, ws_round(sizeof(z) * n * n));
  z* tau = (z*)ws_alloc(c, ws_round(sizeof(z) * n));
  z* p = (z*)ws_alloc(c, ws_round(sizeof(z) * 2 * n));
  double* d = (double*)ws_alloc(c, ws_round(sizeof(double) * n));
  double* e = (double*)ws_alloc(c, ws_round(sizeof(double) * n));
  z* part = (z*)ws_alloc(c, ws_round(sizeof(z) * 2 * TRI_MAX_BLOCKS));
  z* gws = n > TRI_CACHE ? (z*)ws_alloc(c, ws_round(sizeof(z) * 4 * n * TRI_MAX_BLOCKS)) : nullptr;
  unsigned* bar = (unsigned*)ws_alloc(c, 256);
  if (!Hv || !tau || !p || !d || !e || !part || !bar || (n > TRI_CACHE && !gws)) {
    c->ws.top = top;
    return set_err(c, TNT_E_ALLOC, "scratch exhausted (heig_top n=%lld k=%lld)", (long long)n, (long long)k);
  }
  cudaStream_t st = c->stream;
  {
    const double nn = (double)n;
    // Hermitian reduction to tridiagonal form: (16/3) n^3 real FLOPs (4 per complex
    // multiply-add, two rank-2 updates of the trailing block and its matrix-vector product)
    ProfScope ps(c, "heig_tridiag", 16.0 / 3.0 * nn * nn * nn);
    const size_t tri_smem = 4 * TRI_CACHE * sizeof(z);
    static int nsm = 0, occ = 0, rows_dyn_max = 0;
    if (!nsm) {
      TNT_CUDA_TRY(c, cudaFuncSetAttribute(k_tridiag_persistent,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tri_smem));
      TNT_CUDA_TRY(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
      TNT_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tridiag_persistent,
                                                                    TRI_THREADS, tri_smem));
      int optin = 0;
      cudaFuncAttributes fa{};
      TNT_CUDA_TRY(c, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
      TNT_CUDA_TRY(c, cudaFuncGetAttributes(&fa, k_tridiag_rows));
      rows_dyn_max = optin - (int)fa.sharedSizeBytes;
      TNT_CUDA_TRY(c, cudaFuncSetAttribute(k_tridiag_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           rows_dyn_max));
    }
    if (occ < 1) return set_err(c, TNT_E_UNSUPPORTED, "tridiagonal kernel cannot be resident");
    TNT_CUDA_TRY(c, cudaMemsetAsync(bar, 0, 256, st));
    TriArgs ta{G, n, Hv, tau, d, e, p, part, (unsigned*)bar, (int*)(bar + 16), c->d_status,
               gws};
    void* args[] = {&ta};
    // rows resident in shared memory when each block's share and the three vectors fit
    const int nbr = (int)std::min<int64_t>(std::min(nsm, TRI_MAX_BLOCKS), n);
    const int64_t rmax = (n + nbr - 1) / nbr;
    const size_t rows_smem = (size_t)(rmax + 3) * n * sizeof(z);
    int occ_rows = 0;
    if (n <= TRI_ROWS_NMAX && rmax <= TRI_ROWS_MAX && rows_smem <= (size_t)rows_dyn_max)
      TNT_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_rows, k_tridiag_rows,
                                                                    TRI_THREADS, rows_smem));
    if (occ_rows >= 1) {
      TNT_CUDA_TRY(c, cudaLaunchCooperativeKernel((void*)k_tridiag_rows, dim3(nbr),
                                                  dim3(TRI_THREADS), args, rows_smem, st));
    } else {
      const int nb = std::min(nsm, TRI_MAX_BLOCKS);
      TNT_CUDA_TRY(c, cudaLaunchCooperativeKernel((void*)k_tridiag_persistent, dim3(nb),
                                                  dim3(TRI_THREADS), args, tri_smem, st));
    }
    c->launches += 1;
  }
  {
    int h_status = 0;
    TNT_CUDA_TRY(c, cudaMemcpyAsync(&h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    TNT_CUDA_TRY(c, cudaStreamSynchronize(st));
    if (h_status & 2) {
      cudaMemsetAsync(c->d_status, 0, sizeof(int), st);
      c->ws.top = top;
      return set_err(c, TNT_E_TIMEOUT, "tridiagonal reduction: a grid barrier wait expired");
    }
  }
  const int r = heig_finish(c, n, k, Hv, tau, d, e, U, ldu, ev);
  c->ws.top = top;
  return r;
}

// Many small blocks (n <= 256 each): every stage of the eigensolve is one launch over all
// blocks.  blocks[i] = {offset of the n x n block in G (and of its eigenvector columns in
// U, leading dimension n), n, k}; the reduction keeps the reflectors in the blocks' rows.
// ev (device) receives the eigenvalues of all blocks back to back.
int heig_small_blocks(Ctx* c, z* G, const std::vector<SmallEig>& blocks, z* U, double* ev) {
  if (blocks.empty()) return TNT_OK;
  int64_t tot = 0, kt = 0, nk = 0, k2 = 0, nmax = 0;
  for (const SmallEig& b : blocks) {
    if (b.n < 1 || b.n > TRI_CTA_MAX || b.k < 1 || b.k > b.n)
      return set_err(c, TNT_E_INVALID, "small eigensolve block n=%lld k=%lld", (long long)b.n, (long long)b.k);
    tot += b.n;
    kt += b.k;
    nk += b.n * b.k;
    k2 += b.k * b.k;
    nmax = std::max(nmax, b.n);
  }
  const int nb = (int)blocks.size();
  const int cols = BT_COLS;  // sizeof(z) * 256 * 2 fits shared memory
  // host tables: reduction blocks, eigen problems, eigenvalue and back-transformation
  // indices, and the Newton-Schulz task lists with their 16 x 16 tiles
  std::vector<CtaBlk> hc((size_t)nb);
  std::vector<EBlk> he((size_t)nb);
  std::vector<int2> heig, hbt;
  int64_t off = 0, evo = 0, yo = 0, wo = 0, so = 0;
  for (int i = 0; i < nb; ++i) {
    const SmallEig& b = blocks[(size_t)i];
    hc[(size_t)i] = CtaBlk{b.goff, off, (int)b.n};
    he[(size_t)i] = EBlk{b.n, b.k, off, b.goff, evo, yo, wo};
    for (int64_t q = 0; q < b.k; ++q) heig.push_back(make_int2(i, (int)q));
    for (int64_t q = 0; q < b.k; q += cols) hbt.push_back(make_int2(i, (int)q));
    off += b.n;
    evo += b.k;
    yo += b.n * b.k;
    wo += 6 * b.n * b.k;
    so += b.k * b.k;
  }
  const size_t top = c->ws.top;
  double* d = (double*)ws_alloc(c, ws_round(sizeof(double) * tot));
  double* e = (double*)ws_alloc(c, ws_round(sizeof(double) * tot));
  z* tau = (z*)ws_alloc(c, ws_round(sizeof(z) * tot));
  double* tn = (double*)ws_alloc(c, ws_round(sizeof(double) * nb));
  int64_t* nr = (int64_t*)ws_alloc(c, ws_round(sizeof(int64_t) * nb));
  double* work = (double*)ws_alloc(c, ws_round(sizeof(double) * 6 * nk));
  double* Y = (double*)ws_alloc(c, ws_round(sizeof(double) * nk));
  z* U0 = (z*)ws_alloc(c, ws_round(sizeof(z) * nk));
  z* U1 = (z*)ws_alloc(c, ws_round(sizeof(z) * nk));
  z* S = (z*)ws_alloc(c, ws_round(sizeof(z) * k2));
  CtaBlk* dc = (CtaBlk*)ws_alloc(c, ws_round(sizeof(CtaBlk) * nb));
  EBlk* dbl = (EBlk*)ws_alloc(c, ws_round(sizeof(EBlk) * nb));
  int2* deig = (int2*)ws_alloc(c, ws_round(sizeof(int2) * (heig.size() + hbt.size())));
  NsTask* dtask = (NsTask*)ws_alloc(c, ws_round(sizeof(NsTask) * 4 * nb));
  // tiles of the four task lists (S = X^H X and X S, twice)
  std::vector<NsTask> ht;
  std::vector<int4> htile[4];
  for (int step = 0; step < 2; ++step) {
    for (int i = 0; i < nb; ++i) {
      const SmallEig& b = blocks[(size_t)i];
      const EBlk& B = he[(size_t)i];
      z* X = (step == 0 ? U0 : U1) + B.yo;                      // n x k, ld k
      z* Xn = (step == 0) ? U1 + B.yo : U + b.goff;             // next X
      const int64_t ldn = (step == 0) ? b.k : b.n;
      NsTask ts{b.k, b.k, b.n, X, 1, b.k, X, b.k, 1, nullptr, b.k, 1, 1};
      NsTask tx{b.n, b.k, b.k, X, b.k, 1, nullptr, b.k, 1, Xn, ldn, 0, 0};
      ht.push_back(ts);
      ht.push_back(tx);
    }
  }
  {  // S offsets per block
    int64_t o = 0;
    for (int i = 0; i < nb; ++i) {
      const int64_t kb = blocks[(size_t)i].k;
      for (int step = 0; step < 2; ++step) {
        ht[(size_t)(step * 2 * nb + 2 * i)].C = S + o;
        ht[(size_t)(step * 2 * nb + 2 * i + 1)].B = S + o;
      }
      o += kb * kb;
    }
  }
  for (int step = 0; step < 2; ++step)
    for (int which = 0; which < 2; ++which) {
      std::vector<int4>& tl = htile[2 * step + which];
      for (int i = 0; i < nb; ++i) {
        const int ti = step * 2 * nb + 2 * i + which;
        const NsTask& t = ht[(size_t)ti];
        for (int64_t m0 = 0; m0 < t.M; m0 += 16)
          for (int64_t n0 = 0; n0 < t.N; n0 += 16) tl.push_back(make_int4(ti, (int)m0, (int)n0, 0));
      }
    }
  size_t ntile_all = 0;
  for (auto& v : htile) ntile_all += v.size();
  int4* dtile = (int4*)ws_alloc(c, ws_round(sizeof(int4) * ntile_all));
  if (!d || !e || !tau || !tn || !nr || !work || !Y || !U0 || !U1 || !S || !dc || !dbl || !deig || !dtask || !dtile) {
    c->ws.top = top;
    return set_err(c, TNT_E_ALLOC, "scratch exhausted (small eigensolves)");
  }
  cudaStream_t st = c->stream;
  heig.insert(heig.end(), hbt.begin(), hbt.end());
  TNT_CUDA_TRY(c, cudaMemcpyAsync(dc, hc.data(), sizeof(CtaBlk) * nb, cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(dbl, he.data(), sizeof(EBlk) * nb, cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(deig, heig.data(), sizeof(int2) * heig.size(), cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(dtask, ht.data(), sizeof(NsTask) * ht.size(), cudaMemcpyHostToDevice, st));
  {
    size_t o = 0;
    for (auto& v : htile) {
      if (!v.empty())
        TNT_CUDA_TRY(c, cudaMemcpyAsync(dtile + o, v.data(), sizeof(int4) * v.size(), cudaMemcpyHostToDevice, st));
      o += v.size();
    }
  }
  {
    double fl = 0;
    for (const SmallEig& b : blocks) fl += 16.0 / 3.0 * (double)b.n * b.n * b.n;
    ProfScope ps(c, "heig_tridiag", fl);
    k_tridiag_cta<<<(unsigned)nb, TRI_CTA_THREADS, 0, st>>>(G, dc, d, e, tau);
    c->launches++;
    TNT_CHECK_LAUNCH(c);
  }
  {
    ProfScope ps(c, "heig_tridiag_eig");
    k_split<<<(unsigned)nb, 32, 0, st>>>(d, e, dbl, tn, nr);
    k_bisect<<<(unsigned)kt, 32, 0, st>>>(d, e, dbl, deig, nr, tn, ev);
    k_inviter<<<(unsigned)kt, IV_THREADS, 0, st>>>(d, e, dbl, deig, nr, ev, tn, work, Y);
    c->launches += 2;
    TNT_CHECK_LAUNCH(c);
  }
  {
    double fl = 0;
    for (const SmallEig& b : blocks) fl += 8.0 * (double)b.n * b.n * b.k;
    ProfScope ps(c, "heig_backtransform", fl);
    const size_t smem = sizeof(z) * nmax * cols;
    TNT_CUDA_TRY(c, cudaFuncSetAttribute(k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_backtransform<<<(unsigned)hbt.size(), 256, smem, st>>>(Y, G, tau, dbl, deig + kt, cols, U0);
    c->launches++;
    TNT_CHECK_LAUNCH(c);
  }
  {  // two Newton-Schulz steps over all blocks: U0 -> U1 -> U
    size_t o = 0;
    for (int q = 0; q < 4; ++q) {
      const int nt = (int)htile[q].size();
      if (nt > 0) {
        k_gemm_tasks<<<(unsigned)std::min(nt, 152 * 8), 256, 0, st>>>(dtask, dtile + o, nt);
        c->launches++;
        TNT_CHECK_LAUNCH(c);
      }
      o += htile[q].size();
    }
  }
  // the host tables die at return: the uploads above must have completed
  TNT_CUDA_TRY(c, cudaStreamSynchronize(st));
  c->ws.top = top;
  return TNT_OK;
}

}  // namespace tnt
