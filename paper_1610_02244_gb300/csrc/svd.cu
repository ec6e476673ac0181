// Truncated SVD of the reshaped two-site tensor (App. B.1.2, Eq. 3), FP64, on the GPU.
//
// M is block diagonal under U(1) labels (App. A.1.1).  Per block q (rows R_q, columns C_q):
//   LEFT  side: G = M_q M_q^H, eigenvectors U_q (orthonormal), X_q = U_q^H M_q,
//               sigma_k = |row k of X_q|              (so X = S V^H without dividing by S)
//   RIGHT side: G = M_q^H M_q, eigenvectors V_q,      Y_q = M_q V_q,
//               sigma_k = |column k of Y_q|           (so Y = U S)
// Only the k_q = min(m_q, n_q, chi_max) leading eigenvectors are candidates (rank bound,
// and no block can contribute more than chi_max kept values); the weight of the values
// never formed is |M_q|_F^2 minus the candidates'.  Taking sigma as a projection norm
// keeps its absolute error at ~eps |M| instead of the sqrt(eps) relative floor of
// sqrt(lambda).  All candidates are then ordered globally (sigma desc, charge asc, index
// asc) and cut by the four rules in one kernel.  Every block is diagonalised by Householder
// tridiagonalisation, bisection and inverse iteration (heig.cu): blocks up to 256 rows are
// reduced together, one CTA each in one launch, larger ones across the whole GPU.
#include <algorithm>
#include <cmath>
#include <map>

#include "tnt_internal.cuh"

namespace tnt {

namespace {

// sigma of each candidate: norm of row (LEFT: rows of X_q) or column (RIGHT: of Y_q)
struct CandBlock {
  int64_t xoff;   // packed X_q / Y_q offset
  int64_t rows, cols;
  int r;          // candidates
  int vbase;      // first index in the global value list
  int by_row;     // 1: sigma_k = |row k|, 0: |column k|
};

// sigma of every candidate, one warp each: blockIdx.y is the charge block, the CTA's
// eight warps take candidates 8 blockIdx.x ..; the sum of |.|^2 over the candidate's row
// (by_row) or column of X, times the block's unscale
__global__ void __launch_bounds__(256) k_cand_sigma(const z* __restrict__ X,
                                                    const CandBlock* __restrict__ cb,
                                                    const double* __restrict__ unscale,
                                                    double* __restrict__ sig) {
  const CandBlock b = cb[blockIdx.y];
  const int k = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= b.r) return;
  double acc = 0;
  if (b.by_row) {
    for (int64_t c = lane; c < b.cols; c += 32) {
      const z v = X[b.xoff + (int64_t)k * b.cols + c];
      acc = fma(v.x, v.x, fma(v.y, v.y, acc));
    }
  } else {
    for (int64_t i = lane; i < b.rows; i += 32) {
      const z v = X[b.xoff + i * b.cols + k];
      acc = fma(v.x, v.x, fma(v.y, v.y, acc));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) sig[b.vbase + k] = sqrt(acc) * unscale[blockIdx.y];
}

// Each gathered block M_q is scaled by the power of two 2^-e_q that brings max |Re|, |Im|
// into [0.5, 1): exact, and it keeps the Gram matrix and its Householder reduction inside
// the normal range whatever the sector's weight (a sector of theta far from the mean
// filling can hold entries many orders below the rest, whose squares would underflow).
// unscale[q] = 2^e_q multiplies every quantity read back from the scaled block.
// The scale needs only the largest exponent field of the block's entries (a normal x with
// biased exponent e has frexp exponent e - 1022): an integer maximum over the high words,
// taken by as many CTAs per block as its size needs (the maximum does not depend on the
// order), then the scaling by 2^-e_q across the GPU.  A block whose entries are all zero,
// subnormal or non-finite is left unscaled.
__global__ void k_block_maxexp(const z* __restrict__ Mp, const int64_t* __restrict__ boff,
                               const int64_t* __restrict__ bsize, unsigned* __restrict__ mexp) {
  const int q = blockIdx.y;
  const int64_t off = boff[q], cnt = bsize[q];
  unsigned mx = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    const z v = Mp[off + i];
    const unsigned ex = ((unsigned)__double2hiint(v.x) >> 20) & 0x7ffu;
    const unsigned ey = ((unsigned)__double2hiint(v.y) >> 20) & 0x7ffu;
    mx = max(mx, max(ex, ey));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(mexp + q, mx);
}
__global__ void k_block_apply(z* __restrict__ Mp, const int64_t* __restrict__ boff,
                              const int64_t* __restrict__ bsize, const unsigned* __restrict__ mexp,
                              double* __restrict__ unscale) {
  const int q = blockIdx.y;
  const unsigned e = mexp[q];
  const int ex = (e == 0u || e == 2047u) ? 0 : (int)e - 1022;
  if (blockIdx.x == 0 && threadIdx.x == 0) unscale[q] = ldexp(1.0, ex);
  if (ex == 0) return;
  const double sc = ldexp(1.0, -ex);
  const int64_t off = boff[q], cnt = bsize[q];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x)
    Mp[off + i] = zscale(Mp[off + i], sc);
}

// dst[r * ldd + c] = src[r * lds + c], r < rows, c < cols
__global__ void k_copy_strided(const z* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                               z* __restrict__ dst, int64_t ldd) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, cc = e % cols;
    dst[r * ldd + cc] = src[r * lds + cc];
  }
}

// -------------------------------------------------------------- global selection
struct SelOut {
  int64_t chi;
  double err, disc, norm2;
  int tie;
};

__global__ void __launch_bounds__(1024) k_select(const double* __restrict__ sig_in,
                                                 const int* __restrict__ blk_in,
                                                 const int* __restrict__ loc_in, int n, int P,
                                                 int64_t chi_max, double a, double rtol,
                                                 double etol, int etype,
                                                 const double* __restrict__ total_norm2,
                                                 int complete,
                                                 double* __restrict__ sig_out,
                                                 int* __restrict__ blk_out,
                                                 int* __restrict__ loc_out,
                                                 SelOut* __restrict__ res) {
  extern __shared__ double sm_sel[];
  double* key = sm_sel;
  int* bk = (int*)(key + P);
  int* lc = bk + P;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    key[i] = (i < n) ? sig_in[i] : -1.0;
    bk[i] = (i < n) ? blk_in[i] : 0x7fffffff;
    lc[i] = (i < n) ? loc_in[i] : 0x7fffffff;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int l = i ^ j;
        if (l > i) {
          bool desc_block = ((i & k) == 0);
          bool i_before = (key[i] > key[l]) ||
                          (key[i] == key[l] && (bk[i] < bk[l] || (bk[i] == bk[l] && lc[i] < lc[l])));
          bool swap = desc_block ? !i_before : i_before;
          if (swap) {
            double tk = key[i]; key[i] = key[l]; key[l] = tk;
            int tb = bk[i]; bk[i] = bk[l]; bk[l] = tb;
            int tl = lc[i]; lc[i] = lc[l]; lc[l] = tl;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sig_out[i] = key[i];
    blk_out[i] = bk[i];
    loc_out[i] = lc[i];
  }
  if (threadIdx.x == 0) {
    const double s0 = n > 0 ? key[0] : 0.0;
    int64_t chi1 = n < chi_max ? n : chi_max;
    int64_t chi2 = n;
    if (a > 0) {
      chi2 = 0;
      while (chi2 < n && key[chi2] >= a) ++chi2;
    }
    int64_t chi3 = n;
    if (s0 > 0) {
      chi3 = 0;
      while (chi3 < n && key[chi3] / s0 >= rtol) ++chi3;
    }
    // the candidates are each block's leading min(rank, chi_max) values; when that cuts a
    // block short, the weight of the values never formed is |M|_F^2 minus the candidates'
    double sumc = 0;
    for (int i = n - 1; i >= 0; --i) sumc += key[i] * key[i];
    const double nrm2 = complete ? sumc : fmax(total_norm2[0], sumc);
    const double unseen = complete ? 0.0 : fmax(0.0, total_norm2[0] - sumc);
    const double nrm = sqrt(nrm2);
    const double inv = nrm > 0 ? 1.0 / nrm : 1.0;
    auto term = [&](double s) {
      double t = s * inv;
      return etype == TNT_TRUNC_1NORM ? fabs(t) : t * t;
    };
    auto errf = [&](double acc) { return etype == TNT_TRUNC_2NORM ? sqrt(acc) : acc; };
    const double acc0 = unseen * inv * inv;  // never formed values, in normalised units
    int64_t chi4 = n;
    double acc = acc0;
    if (!(errf(acc) < etol)) chi4 = n;
    for (int keep = n - 1; keep >= 0 && errf(acc) < etol; --keep) {
      acc += term(key[keep]);
      if (errf(acc) < etol) chi4 = keep; else break;
    }
    int64_t chi = chi1;
    if (chi2 < chi) chi = chi2;
    if (chi3 < chi) chi = chi3;
    if (chi4 < chi) chi = chi4;
    if (chi < 1) chi = 1;
    if (chi > n) chi = n;
    double e = acc0, dsc = unseen;
    for (int i = n - 1; i >= chi; --i) {
      e += term(key[i]);
      dsc += key[i] * key[i];
    }
    res->chi = chi;
    res->err = errf(e);
    res->disc = dsc;
    res->norm2 = nrm2;
    res->tie = (chi < n) && (key[chi - 1] - key[chi] < 1e-10 * s0);
  }
}

// -------------------------------------------------------------- output scatter
// One bond index k per blockIdx.y.  LEFT: U[rows[r]][k] = Vq[r][loc] (r < m_q), and
// X[k][cols[c]] = scale * Xq[loc][c].  RIGHT: X[k][cols[c]] = conj(Vq[c][loc]) and
// U[rows[r]][k] = scale * Yq[r][loc].
struct KeptIdx {
  int64_t voff, vld;     // eigenvector block (ld = Gram dim)
  int64_t xoff, xld;     // X_q (LEFT: r x n_q, ld n_q) or Y_q (RIGHT: m_q x r, ld r)
  int64_t roff, nr;      // rows list slice
  int64_t coff, nc;      // cols list slice
  int loc;
  int blk;               // block index (its unscale factor)
};

__global__ void k_scatter(const z* __restrict__ Vp, const z* __restrict__ Xp,
                          const KeptIdx* __restrict__ kept, const int64_t* __restrict__ rows,
                          const int64_t* __restrict__ cols, const double* __restrict__ unscale,
                          int side, double scale0, int64_t chi, int64_t n_total,
                          z* __restrict__ U, z* __restrict__ X) {
  const int64_t k = blockIdx.y;
  const KeptIdx kd = kept[k];
  const double scale = scale0 * unscale[kd.blk];
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < kd.nr;
       r += (int64_t)gridDim.x * blockDim.x) {
    z v;
    if (side == TNT_SVD_LEFT) v = Vp[kd.voff + r * kd.vld + kd.loc];
    else v = zscale(Xp[kd.xoff + r * kd.xld + kd.loc], scale);
    U[rows[kd.roff + r] * chi + k] = v;
  }
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < kd.nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    z v;
    if (side == TNT_SVD_LEFT) v = zscale(Xp[kd.xoff + (int64_t)kd.loc * kd.xld + c], scale);
    else v = zconj(Vp[kd.voff + c * kd.vld + kd.loc]);
    X[k * n_total + cols[kd.coff + c]] = v;
  }
}

// automatic blocking: Mz = M with |M_ij| <= tol set to zero, mask bit j of row i's word
// j / 32 set where |M_ij| > tol; one thread per 32-column word
__global__ void k_autoblock(const z* __restrict__ M, int64_t m, int64_t n, double tol,
                            z* __restrict__ Mz, uint32_t* __restrict__ mask) {
  const int64_t W = (n + 31) / 32;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m * W;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / W, w = t % W;
    uint32_t bits = 0;
    for (int b = 0; b < 32; ++b) {
      const int64_t j = w * 32 + b;
      if (j >= n) break;
      const z v = M[i * n + j];
      const bool keep = sqrt(v.x * v.x + v.y * v.y) > tol;
      Mz[i * n + j] = keep ? v : zmk(0, 0);
      bits |= keep ? (1u << b) : 0u;
    }
    mask[t] = bits;
  }
}

unsigned gridn(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return (unsigned)b;
}
}  // namespace

// ==================================================================== truncated SVD
// connected components of the bipartite non-zero pattern (rows 0..m-1, columns m..m+n-1;
// bit j % 32 of mask[i * W + j / 32] marks a non-zero M_ij, W = ceil(n / 32)), union-find
// with path halving; a component is numbered by its first row, components of columns alone
// follow in column order.  Returns the number of components.
int64_t autoblock_components(int64_t m, int64_t n, const uint32_t* mask, int64_t* row_q,
                             int64_t* col_q) {
  const int64_t W = (n + 31) / 32;
  std::vector<int64_t> parent((size_t)(m + n));
  for (int64_t v = 0; v < m + n; ++v) parent[(size_t)v] = v;
  auto find = [&](int64_t v) {
    while (parent[(size_t)v] != v) {
      parent[(size_t)v] = parent[(size_t)parent[(size_t)v]];
      v = parent[(size_t)v];
    }
    return v;
  };
  for (int64_t i = 0; i < m; ++i)
    for (int64_t w = 0; w < W; ++w) {
      uint32_t bits = mask[(size_t)(i * W + w)];
      while (bits) {
        const int b = __builtin_ctz(bits);
        bits &= bits - 1;
        if (w * 32 + b >= n) break;
        const int64_t a = find(i), r = find(m + w * 32 + b);
        if (a != r) parent[(size_t)std::max(a, r)] = std::min(a, r);
      }
    }
  std::vector<int64_t> id((size_t)(m + n), -1);
  int64_t next = 0;
  for (int64_t i = 0; i < m; ++i) {
    const int64_t r = find(i);
    if (id[(size_t)r] < 0) id[(size_t)r] = next++;
    row_q[i] = id[(size_t)r];
  }
  for (int64_t j = 0; j < n; ++j) {
    const int64_t r = find(m + j);
    if (id[(size_t)r] < 0) id[(size_t)r] = next++;
    col_q[j] = id[(size_t)r];
  }
  return next;
}

static size_t autoblock_bytes(int64_t m, int64_t n) {
  return ws_round(sizeof(z) * (size_t)m * n) + ws_round(sizeof(uint32_t) * (size_t)m * ((n + 31) / 32));
}

size_t svd_scratch_bound(int64_t m, int64_t n) {
  const size_t mx = (size_t)std::max(m, n), mn = (size_t)std::min(m, n);
  // the eigen phase of the small blocks (Gram side <= 256, every eigenpair formed): per
  // block n k <= 256 n of work, iterates, two eigenvector copies and k^2 coefficients
  const size_t small_eig = (6 * 8 + 8 + 2 * 16 + 16) * 256 * mx + (size_t)(1 << 20);
  // the tail pass: its Gram matrices and eigenvectors (sum t^2 <= mx mn each), one rotation
  // buffer (<= mx mn), eigenvalues
  const size_t tail = 3 * 16 * mx * mn + 8 * std::max<size_t>(mx * mn, 8192);
  return autoblock_bytes(m, n) + 8 * (size_t)(m + n) + 2 * 16 * (size_t)m * n + 2 * 16 * mx * mx + 6 * 8 * mx +
         sizeof(KeptIdx) * mx + 12 * 8192 + tail +
         std::max(heig_scratch_bound((int64_t)mx, (int64_t)mx), small_eig) + (size_t)(4 << 20);
}

namespace {
// one charge block of the truncated SVD (host tables)
struct Blk {
  int64_t q, mq, nq, g, r, k;
  int64_t roff, coff, moff, goff, xoff;
};
// Second pass over each block's tail.  An eigenvector of the Gram matrix whose eigenvalue
// lies at the Gram matrix's rounding level (or below the split of its tridiagonal form) is
// only known to lie in the right subspace: its projection norm mixes the tiny singular
// values of that subspace with the Gram matrix's rounding, which is ~sqrt(eps) |M| rather
// than eps |M|.  So the candidates of a block whose sigma is below TAIL_REL times the
// block's largest (a suffix of the candidate list, which runs in eigenvalue order) are
// diagonalised once more, from their own projections: LEFT, H = X_t X_t^H of the tail rows
// X_t = U_t^H M_q; RIGHT, H = Y_t^H Y_t of the tail columns Y_t = M_q V_t.  H carries the
// tail's own scale, so its eigenvectors W resolve the tail's singular values down to about
// eps |M|; U_t <- U_t W (V_t <- V_t W) and X_t <- W^H X_t (Y_t <- Y_t W) rotate the
// candidates within the tail subspace, keeping them orthonormal, and the projection norms
// are taken again.
// Blocks of up to 256 rows are reduced either together, one CTA (one SM) each, or one by
// one by the cooperative kernel across the GPU.  On one SM a block costs about
// 1.3e-9 n^3 s (its 4 n^3 FP64 FMAs at two per clock, plus per-column overhead); across
// the GPU about 15 us per column, plus 6.4e-12 n^3 s of FP64 work and 0.5 ms for its own
// eigenvalue, vector and back-transformation launches.  The batch takes as long as its
// largest block, or its total over the SMs.  The largest blocks move to the cooperative
// path while that shortens the estimate: a lone 256-row block (the tail of a truncated
// SVD whose spectrum falls fast) takes about 4 ms there against about 20 ms on one SM.
std::vector<char> route_coop(const std::vector<int64_t>& ns, int nsm) {
  auto t_cta = [](double n) { return 1.3e-9 * n * n * n; };
  auto t_coop = [](double n) { return 15e-6 * n + 6.4e-12 * n * n * n + 5e-4; };
  std::vector<int> ord(ns.size());
  for (size_t i = 0; i < ns.size(); ++i) ord[i] = (int)i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return ns[(size_t)a] > ns[(size_t)b]; });
  auto batch = [&](size_t from) {  // the one-CTA batch over ord[from..]
    double mx = 0, sum = 0;
    for (size_t i = from; i < ord.size(); ++i) {
      const double t = t_cta((double)ns[(size_t)ord[i]]);
      mx = std::max(mx, t);
      sum += t;
    }
    return std::max(mx, sum / std::max(1, nsm));
  };
  double best = batch(0), acc = 0;
  size_t moved = 0;
  for (size_t i = 0; i < ord.size(); ++i) {
    acc += t_coop((double)ns[(size_t)ord[i]]);
    const double cand = acc + batch(i + 1);
    if (cand < best) {
      best = cand;
      moved = i + 1;
    }
  }
  std::vector<char> coop(ns.size(), 0);
  for (size_t i = 0; i < moved; ++i) coop[(size_t)ord[i]] = 1;
  return coop;
}

int sm_count(Ctx* c) {
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) nsm = 1;
  return nsm;
}

constexpr double TAIL_REL = 1e-4;

struct TailBlk {
  int b;
  int64_t t0, t, toff;
};

int refine_tails(Ctx* c, int side, const std::vector<Blk>& bl, z* Vp, z* Xp,
                 const CandBlock* d_cb, const double* d_unscale, double* d_sig, int64_t ntot) {
  cudaStream_t st = c->stream;
  std::vector<double> hs((size_t)ntot);
  TNT_CUDA_TRY(c, cudaMemcpyAsync(hs.data(), d_sig, sizeof(double) * ntot, cudaMemcpyDeviceToHost, st));
  TNT_CUDA_TRY(c, cudaStreamSynchronize(st));
  std::vector<TailBlk> tb;
  int64_t gt = 0, vbase = 0, tmpmax = 0;
  for (int b = 0; b < (int)bl.size(); ++b) {
    const Blk& B = bl[(size_t)b];
    double mx = 0;
    for (int64_t i = 0; i < B.k; ++i) mx = std::max(mx, hs[(size_t)(vbase + i)]);
    int64_t t0 = B.k;
    while (t0 > 0 && !(hs[(size_t)(vbase + t0 - 1)] >= TAIL_REL * mx)) --t0;
    const int64_t t = B.k - t0;
    if (t >= 2 && mx > 0) {
      tb.push_back(TailBlk{b, t0, t, gt});
      gt += t * t;
      const int64_t rows_x = (side == TNT_SVD_LEFT) ? t : B.mq;
      const int64_t cols_x = (side == TNT_SVD_LEFT) ? B.nq : t;
      tmpmax = std::max(tmpmax, std::max(B.g * t, rows_x * cols_x));
    }
    vbase += B.k;
  }
  if (tb.empty()) return TNT_OK;
  const size_t top = c->ws.top;
  z* H = (z*)ws_alloc(c, ws_round(sizeof(z) * gt));
  z* W = (z*)ws_alloc(c, ws_round(sizeof(z) * gt));
  z* tmp = (z*)ws_alloc(c, ws_round(sizeof(z) * tmpmax));
  double* ev = (double*)ws_alloc(c, ws_round(sizeof(double) * (gt > 8192 ? gt : 8192)));
  if (!H || !W || !tmp || !ev) {
    c->ws.top = top;
    return set_err(c, TNT_E_ALLOC, "scratch exhausted (SVD tail pass)");
  }
  // tail Gram matrices
  for (const TailBlk& T : tb) {
    const Blk& B = bl[(size_t)T.b];
    ZGemm g{};
    g.batch = 1;
    g.alpha = zmk(1, 0);
    g.beta = zmk(0, 0);
    g.M = T.t; g.N = T.t;
    g.C = H + T.toff; g.c_rs = T.t;
    if (side == TNT_SVD_LEFT) {  // H = X_t X_t^H, X_t rows t0.. of X_q (ld n_q)
      const z* Xt = Xp + B.xoff + T.t0 * B.nq;
      g.K = B.nq;
      g.A = Xt; g.a_rs = B.nq; g.a_cs = 1;
      g.B = Xt; g.b_rs = 1; g.b_cs = B.nq; g.conj_b = 1;
    } else {  // H = Y_t^H Y_t, Y_t columns t0.. of Y_q (ld k)
      const z* Yt = Xp + B.xoff + T.t0;
      g.K = B.mq;
      g.A = Yt; g.a_rs = 1; g.a_cs = B.k; g.conj_a = 1;
      g.B = Yt; g.b_rs = B.k; g.b_cs = 1;
    }
    TNT_TRY(zgemm(c, g));
  }
  // eigenvectors of every tail Gram matrix (all of them, descending)
  {
    std::vector<int64_t> ns;
    for (const TailBlk& T : tb) ns.push_back(T.t <= 256 ? T.t : 0);
    const std::vector<char> coop = route_coop(ns, sm_count(c));
    std::vector<SmallEig> small;
    for (size_t i = 0; i < tb.size(); ++i)
      if (tb[i].t <= 256 && !coop[i]) small.push_back(SmallEig{tb[i].toff, tb[i].t, tb[i].t});
    TNT_TRY(heig_small_blocks(c, H, small, W, ev));
    for (size_t i = 0; i < tb.size(); ++i) {
      const TailBlk& T = tb[i];
      if (T.t > 256 || coop[i]) TNT_TRY(heig_top(c, H + T.toff, T.t, T.t, W + T.toff, T.t, ev));
    }
  }
  // rotate the tail candidates within their subspace
  for (const TailBlk& T : tb) {
    const Blk& B = bl[(size_t)T.b];
    z* Wt = W + T.toff;
    {  // eigenvectors: U_t (or V_t), g x t at column t0 of the block (ld g) <- U_t W
      ZGemm g{};
      g.batch = 1; g.alpha = zmk(1, 0); g.beta = zmk(0, 0);
      g.M = B.g; g.N = T.t; g.K = T.t;
      g.A = Vp + B.goff + T.t0; g.a_rs = B.g; g.a_cs = 1;
      g.B = Wt; g.b_rs = T.t; g.b_cs = 1;
      g.C = tmp; g.c_rs = T.t;
      TNT_TRY(zgemm(c, g));
      k_copy_strided<<<gridn(B.g * T.t), 256, 0, st>>>(tmp, B.g, T.t, T.t, Vp + B.goff + T.t0, B.g);
      c->launches++;
    }
    ZGemm g{};
    g.batch = 1; g.alpha = zmk(1, 0); g.beta = zmk(0, 0);
    if (side == TNT_SVD_LEFT) {  // X_t <- W^H X_t  (t x n_q, contiguous rows)
      z* Xt = Xp + B.xoff + T.t0 * B.nq;
      g.M = T.t; g.N = B.nq; g.K = T.t;
      g.A = Wt; g.a_rs = 1; g.a_cs = T.t; g.conj_a = 1;
      g.B = Xt; g.b_rs = B.nq; g.b_cs = 1;
      g.C = tmp; g.c_rs = B.nq;
      TNT_TRY(zgemm(c, g));
      TNT_CUDA_TRY(c, cudaMemcpyAsync(Xt, tmp, sizeof(z) * T.t * B.nq, cudaMemcpyDeviceToDevice, st));
    } else {  // Y_t <- Y_t W  (m_q x t at column t0, ld k)
      z* Yt = Xp + B.xoff + T.t0;
      g.M = B.mq; g.N = T.t; g.K = T.t;
      g.A = Yt; g.a_rs = B.k; g.a_cs = 1;
      g.B = Wt; g.b_rs = T.t; g.b_cs = 1;
      g.C = tmp; g.c_rs = T.t;
      TNT_TRY(zgemm(c, g));
      k_copy_strided<<<gridn(B.mq * T.t), 256, 0, st>>>(tmp, B.mq, T.t, T.t, Yt, B.k);
      c->launches++;
    }
  }
  TNT_CHECK_LAUNCH(c);
  {
    int64_t rmax = 1;
    for (const Blk& B : bl) rmax = std::max<int64_t>(rmax, B.k);
    k_cand_sigma<<<dim3((unsigned)((rmax + 7) / 8), (unsigned)bl.size()), 256, 0, st>>>(Xp, d_cb, d_unscale, d_sig);
  }
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  c->ws.top = top;
  return TNT_OK;
}
}  // namespace

int svd_trunc_impl(Ctx* c, const z* M, int64_t m, int64_t n, const int64_t* h_rq,
                   const int64_t* h_cq, int side, int renorm, z* U, z* X, double* h_S,
                   int64_t* h_bq, tnt_trunc_result* res) {
  const tnt_params& P = c->params;
  TNT_TRY(ws_reserve(c, c->ws.top + svd_scratch_bound(m, n)));
  // ---- automatic blocking of an unlabelled matrix (Sec. 6): zero |M_ij| <= tol, then the
  // connected components of the non-zero pattern are the blocks (union-find on the host
  // over the bit mask; a component is numbered by its first row, then columns alone)
  std::vector<int64_t> arq, acq;
  bool unlabelled = (h_rq == nullptr);
  if (!unlabelled) {
    unlabelled = true;
    for (int64_t i = 1; i < m && unlabelled; ++i) unlabelled = (h_rq[i] == h_rq[0]);
    for (int64_t j = 0; j < n && unlabelled; ++j) unlabelled = (h_cq[j] == h_rq[0]);
  }
  if (unlabelled && c->svd_zero_tol >= 0) {
    const int64_t W = (n + 31) / 32;
    z* Mz = (z*)ws_alloc(c, ws_round(sizeof(z) * (size_t)m * n));
    uint32_t* dmask = (uint32_t*)ws_alloc(c, ws_round(sizeof(uint32_t) * (size_t)m * W));
    if (!Mz || !dmask) return set_err(c, TNT_E_ALLOC, "scratch exhausted (automatic blocking)");
    k_autoblock<<<gridn(m * W), 256, 0, c->stream>>>(M, m, n, c->svd_zero_tol, Mz, dmask);
    c->launches++;
    TNT_CHECK_LAUNCH(c);
    std::vector<uint32_t> hm((size_t)(m * W));
    TNT_CUDA_TRY(c, cudaMemcpyAsync(hm.data(), dmask, sizeof(uint32_t) * hm.size(), cudaMemcpyDeviceToHost, c->stream));
    TNT_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    arq.resize((size_t)m);
    acq.resize((size_t)n);
    autoblock_components(m, n, hm.data(), arq.data(), acq.data());
    M = Mz;
    h_rq = arq.data();
    h_cq = acq.data();
  }
  // ---- block structure (host, integer only)
  std::map<int64_t, std::pair<std::vector<int64_t>, std::vector<int64_t>>> blocks;
  for (int64_t i = 0; i < m; ++i) blocks[h_rq ? h_rq[i] : 0].first.push_back(i);
  for (int64_t j = 0; j < n; ++j) {
    int64_t q = h_cq ? h_cq[j] : 0;
    auto it = blocks.find(q);
    if (it != blocks.end()) it->second.second.push_back(j);
  }
  // candidates per block: its leading min(rank, chi_max) values (all of them for the
  // 1-norm error, which cannot be completed from |M|_F)
  const bool all_values = (P.trunc_type == TNT_TRUNC_1NORM);

  bool complete = true;
  std::vector<Blk> bl;
  std::vector<int64_t> rows_all, cols_all;
  int64_t mtot = 0, gtot = 0, xtot = 0, ntot_vals = 0;
  for (auto& kv : blocks) {
    const auto& R = kv.second.first;
    const auto& Cc = kv.second.second;
    if (R.empty() || Cc.empty()) continue;
    Blk b;
    b.q = kv.first;
    b.mq = (int64_t)R.size();
    b.nq = (int64_t)Cc.size();
    b.g = (side == TNT_SVD_LEFT) ? b.mq : b.nq;
    b.r = std::min(b.mq, b.nq);
    const int64_t kb = all_values ? b.r : std::min<int64_t>(b.r, P.chi_max);
    // every eigenpair of the Gram matrix where that costs little more than the candidates
    // (small blocks, or a Gram side within 1.25 times the candidate bound): rounding-level
    // eigenvalues come from the split of the tridiagonal matrix at no iteration cost, and
    // the block's weight is then accounted exactly instead of as |M_q|^2 minus the
    // candidates' (which cannot resolve weights below eps |M_q|^2)
    b.k = (b.g <= 256 || 4 * b.g <= 5 * kb) ? b.g : kb;
    if (b.k < b.r) complete = false;
    b.roff = (int64_t)rows_all.size();
    b.coff = (int64_t)cols_all.size();
    rows_all.insert(rows_all.end(), R.begin(), R.end());
    cols_all.insert(cols_all.end(), Cc.begin(), Cc.end());
    b.moff = mtot;
    mtot += b.mq * b.nq;
    b.goff = gtot;
    gtot += b.g * b.g;
    b.xoff = xtot;
    xtot += (side == TNT_SVD_LEFT) ? b.k * b.nq : b.mq * b.k;
    ntot_vals += b.k;
    bl.push_back(b);
  }
  const int nb = (int)bl.size();
  if (nb == 0 || ntot_vals == 0) return set_err(c, TNT_E_INVALID, "SVD: no charge block has both rows and columns");
  if (ntot_vals > 8192) return set_err(c, TNT_E_UNSUPPORTED, "SVD: %lld candidate values > 8192", (long long)ntot_vals);

  // ---- scratch
  int P2 = 1;
  while (P2 < ntot_vals) P2 <<= 1;
  int64_t* d_rows = (int64_t*)ws_alloc(c, ws_round(sizeof(int64_t) * rows_all.size()));
  int64_t* d_cols = (int64_t*)ws_alloc(c, ws_round(sizeof(int64_t) * cols_all.size()));
  z* Mp = (z*)ws_alloc(c, ws_round(sizeof(z) * mtot));
  z* Gp = (z*)ws_alloc(c, ws_round(sizeof(z) * gtot));
  z* Vp = (z*)ws_alloc(c, ws_round(sizeof(z) * gtot));
  z* Xp = (z*)ws_alloc(c, ws_round(sizeof(z) * xtot));
  double* d_sig = (double*)ws_alloc(c, ws_round(sizeof(double) * ntot_vals));
  int* d_blk = (int*)ws_alloc(c, ws_round(sizeof(double) * ntot_vals));
  int* d_loc = (int*)ws_alloc(c, ws_round(sizeof(double) * ntot_vals));
  double* d_sig_s = (double*)ws_alloc(c, ws_round(sizeof(double) * ntot_vals));
  int* d_blk_s = (int*)ws_alloc(c, ws_round(sizeof(double) * ntot_vals));
  int* d_loc_s = (int*)ws_alloc(c, ws_round(sizeof(double) * ntot_vals));
  SelOut* d_sel = (SelOut*)ws_alloc(c, ws_round(sizeof(SelOut)));
  CandBlock* d_cb = (CandBlock*)ws_alloc(c, ws_round(sizeof(CandBlock) * nb));
  int64_t* d_goff = (int64_t*)ws_alloc(c, ws_round(sizeof(int64_t) * nb));
  int* d_gdim = (int*)ws_alloc(c, ws_round(sizeof(int64_t) * nb));
  double* d_ev = (double*)ws_alloc(c, ws_round(sizeof(double) * 8192));
  double* d_tot = (double*)ws_alloc(c, ws_round(sizeof(double)));
  double* d_unscale = (double*)ws_alloc(c, ws_round(sizeof(double) * nb));
  unsigned* d_mexp = (unsigned*)ws_alloc(c, ws_round(sizeof(unsigned) * nb));
  int64_t* d_boff = (int64_t*)ws_alloc(c, ws_round(sizeof(int64_t) * 2 * nb));
  if (!d_unscale || !d_mexp || !d_boff) return set_err(c, TNT_E_ALLOC, "scratch exhausted (svd)");
  if (!d_rows || !d_cols || !Mp || !Gp || !Vp || !Xp || !d_sig || !d_blk || !d_loc || !d_sig_s ||
      !d_blk_s || !d_loc_s || !d_sel || !d_cb || !d_goff || !d_gdim || !d_ev || !d_tot)
    return set_err(c, TNT_E_ALLOC, "scratch exhausted (svd)");

  // ---- host tables -> device (one synchronous upload of small integer tables)
  std::vector<CandBlock> hcb(nb);
  std::vector<int64_t> hgoff(nb);
  std::vector<int> hgdim(nb), hblk(ntot_vals), hloc(ntot_vals);
  std::vector<int64_t> hboff(2 * (size_t)nb);
  {
    int v = 0;
    for (int b = 0; b < nb; ++b) {
      hcb[b].xoff = bl[b].xoff;
      hcb[b].rows = (side == TNT_SVD_LEFT) ? bl[b].k : bl[b].mq;
      hcb[b].cols = (side == TNT_SVD_LEFT) ? bl[b].nq : bl[b].k;
      hcb[b].r = (int)bl[b].k;
      hcb[b].vbase = v;
      hcb[b].by_row = (side == TNT_SVD_LEFT);
      hgoff[b] = bl[b].goff;
      hgdim[b] = (int)bl[b].g;
      hboff[b] = bl[b].moff;
      hboff[nb + b] = bl[b].mq * bl[b].nq;
      for (int k = 0; k < bl[b].k; ++k, ++v) {
        hblk[v] = b;
        hloc[v] = k;
      }
    }
  }
  cudaStream_t st = c->stream;
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_rows, rows_all.data(), sizeof(int64_t) * rows_all.size(), cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_cols, cols_all.data(), sizeof(int64_t) * cols_all.size(), cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_cb, hcb.data(), sizeof(CandBlock) * nb, cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_goff, hgoff.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_gdim, hgdim.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_blk, hblk.data(), sizeof(int) * ntot_vals, cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_loc, hloc.data(), sizeof(int) * ntot_vals, cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_boff, hboff.data(), sizeof(int64_t) * 2 * nb, cudaMemcpyHostToDevice, st));

  // ---- gather blocks, |M|_F^2 (unscaled), scale each block, Gram matrices
  for (int b = 0; b < nb; ++b) {
    const Blk& B = bl[b];
    TNT_TRY(gather2d(c, M, n, d_rows + B.roff, B.mq, d_cols + B.coff, B.nq, Mp + B.moff, B.nq, 0));
  }
  TNT_TRY(vec_norm2(c, Mp, mtot, d_tot));
  {
    int64_t mxcnt = 1;
    for (int b = 0; b < nb; ++b) mxcnt = std::max<int64_t>(mxcnt, (int64_t)bl[b].mq * bl[b].nq);
    const unsigned per = (unsigned)std::min<int64_t>(64, (mxcnt + 4095) / 4096);  // CTAs per block
    TNT_CUDA_TRY(c, cudaMemsetAsync(d_mexp, 0, sizeof(unsigned) * nb, st));
    k_block_maxexp<<<dim3(per, nb), 256, 0, st>>>(Mp, d_boff, d_boff + nb, d_mexp);
    k_block_apply<<<dim3(per, nb), 256, 0, st>>>(Mp, d_boff, d_boff + nb, d_mexp, d_unscale);
    c->launches += 2;
  }
  TNT_CHECK_LAUNCH(c);
  for (int b = 0; b < nb; ++b) {
    const Blk& B = bl[b];
    ZGemm g{};
    g.batch = 1;
    g.alpha = zmk(1, 0);
    g.beta = zmk(0, 0);
    g.C = Gp + B.goff;
    g.c_rs = B.g;
    if (side == TNT_SVD_LEFT) {  // G = M M^H
      g.M = B.mq; g.N = B.mq; g.K = B.nq;
      g.A = Mp + B.moff; g.a_rs = B.nq; g.a_cs = 1;
      g.B = Mp + B.moff; g.b_rs = 1; g.b_cs = B.nq; g.conj_b = 1;
    } else {  // G = M^H M
      g.M = B.nq; g.N = B.nq; g.K = B.mq;
      g.A = Mp + B.moff; g.a_rs = 1; g.a_cs = B.nq; g.conj_a = 1;
      g.B = Mp + B.moff; g.b_rs = B.nq; g.b_cs = 1;
    }
    g.lower_only = 1;  // G is Hermitian: form the lower tiles, mirror the rest
    TNT_TRY(zgemm(c, g));
    TNT_TRY(herm_mirror(c, Gp + B.goff, B.g));
  }
  // ---- eigensolves: blocks up to 256 rows reduced together (one CTA each, one launch),
  // larger ones, and small ones that would hold the batch back (route_coop), one by one
  // across the whole GPU
  {
    std::vector<int64_t> ns;
    for (int b = 0; b < nb; ++b) ns.push_back(bl[b].g <= 256 ? bl[b].g : 0);
    const std::vector<char> coop = route_coop(ns, sm_count(c));
    std::vector<SmallEig> small;
    for (int b = 0; b < nb; ++b)
      if (bl[b].g <= 256 && !coop[(size_t)b]) small.push_back(SmallEig{bl[b].goff, bl[b].g, bl[b].k});
    TNT_TRY(heig_small_blocks(c, Gp, small, Vp, d_ev));
    for (int b = 0; b < nb; ++b) {
      if (bl[b].g <= 256 && !coop[(size_t)b]) continue;
      const Blk& B = bl[b];
      if (B.g > 8192) return set_err(c, TNT_E_UNSUPPORTED, "SVD block of dim %lld > 8192", (long long)B.g);
      TNT_TRY(heig_top(c, Gp + B.goff, B.g, B.k, Vp + B.goff, B.g, d_ev));
    }
  }
  // ---- candidate products and their norms
  for (int b = 0; b < nb; ++b) {
    const Blk& B = bl[b];
    ZGemm g{};
    g.batch = 1;
    g.alpha = zmk(1, 0);
    g.beta = zmk(0, 0);
    if (side == TNT_SVD_LEFT) {  // X_q = U_q[:, :k]^H M_q  (k x n_q)
      g.M = B.k; g.N = B.nq; g.K = B.mq;
      g.A = Vp + B.goff; g.a_rs = 1; g.a_cs = B.g; g.conj_a = 1;
      g.B = Mp + B.moff; g.b_rs = B.nq; g.b_cs = 1;
      g.C = Xp + B.xoff; g.c_rs = B.nq;
    } else {  // Y_q = M_q V_q[:, :k]  (m_q x k)
      g.M = B.mq; g.N = B.k; g.K = B.nq;
      g.A = Mp + B.moff; g.a_rs = B.nq; g.a_cs = 1;
      g.B = Vp + B.goff; g.b_rs = B.g; g.b_cs = 1;
      g.C = Xp + B.xoff; g.c_rs = B.k;
    }
    TNT_TRY(zgemm(c, g));
  }
  {
    int64_t rmax = 1;
    for (int b = 0; b < nb; ++b) rmax = std::max<int64_t>(rmax, bl[b].k);
    k_cand_sigma<<<dim3((unsigned)((rmax + 7) / 8), (unsigned)nb), 256, 0, st>>>(Xp, d_cb, d_unscale, d_sig);
  }
  c->launches++;
  TNT_TRY(refine_tails(c, side, bl, Vp, Xp, d_cb, d_unscale, d_sig, ntot_vals));
  // ---- global order and the four rules
  {
    size_t smem = (size_t)P2 * (sizeof(double) + 2 * sizeof(int));
    TNT_CUDA_TRY(c, cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // never more than the blocks' rank bounds (at most min(m, n), the callers' capacity),
    // whatever the number of candidates formed
    int64_t rank_total = 0;
    for (const Blk& B : bl) rank_total += B.r;
    k_select<<<1, 1024, smem, st>>>(d_sig, d_blk, d_loc, (int)ntot_vals, P2,
                                    std::min<int64_t>(P.chi_max, rank_total), P.trunc_abs,
                                    P.trunc_rel, P.trunc_err, P.trunc_type, d_tot, complete ? 1 : 0,
                                    d_sig_s, d_blk_s, d_loc_s, d_sel);
    c->launches++;
    TNT_CHECK_LAUNCH(c);
  }
  SelOut sel;
  std::vector<double> hs(ntot_vals);
  std::vector<int> hb(ntot_vals), hl(ntot_vals);
  TNT_CUDA_TRY(c, cudaMemcpyAsync(&sel, d_sel, sizeof(SelOut), cudaMemcpyDeviceToHost, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(hs.data(), d_sig_s, sizeof(double) * ntot_vals, cudaMemcpyDeviceToHost, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(hb.data(), d_blk_s, sizeof(int) * ntot_vals, cudaMemcpyDeviceToHost, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(hl.data(), d_loc_s, sizeof(int) * ntot_vals, cudaMemcpyDeviceToHost, st));
  TNT_CUDA_TRY(c, cudaStreamSynchronize(st));
  const int64_t chi = sel.chi;
  if (chi < 1 || chi > ntot_vals) return set_err(c, TNT_E_NAN, "SVD selection returned chi = %lld of %lld", (long long)chi, (long long)ntot_vals);
  for (int64_t k = 0; k < ntot_vals; ++k)  // report the block of a non-finite value first
    if (!std::isfinite(hs[k]) && hb[k] >= 0 && hb[k] < nb)
      return set_err(c, TNT_E_NAN, "SVD of %lld x %lld (%d blocks): value %g in block %d (%lld x %lld, Gram %lld, candidate %d of %lld)",
                     (long long)m, (long long)n, nb, hs[k], hb[k], (long long)bl[hb[k]].mq,
                     (long long)bl[hb[k]].nq, (long long)bl[hb[k]].g, hl[k], (long long)bl[hb[k]].k);
  for (int64_t k = 0; k < ntot_vals; ++k)  // a non-finite value sorts anywhere: never index with it
    if (!std::isfinite(hs[k]) || hb[k] < 0 || hb[k] >= nb || hl[k] < 0 || hl[k] >= bl[hb[k]].k)
      return set_err(c, TNT_E_NAN,
                     "SVD of %lld x %lld (%d blocks): non-finite or misplaced value %g at sorted index "
                     "%lld (block %d, %lld x %lld, Gram %lld, candidate %d of %lld)",
                     (long long)m, (long long)n, nb, hs[k], (long long)k, hb[k],
                     (hb[k] >= 0 && hb[k] < nb) ? (long long)bl[hb[k]].mq : -1LL,
                     (hb[k] >= 0 && hb[k] < nb) ? (long long)bl[hb[k]].nq : -1LL,
                     (hb[k] >= 0 && hb[k] < nb) ? (long long)bl[hb[k]].g : -1LL, hl[k],
                     (hb[k] >= 0 && hb[k] < nb) ? (long long)bl[hb[k]].k : -1LL);
  // ---- bond order: charge ascending (block index), then sigma descending
  std::vector<int> order(chi);
  for (int64_t k = 0; k < chi; ++k) order[k] = (int)k;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hb[x] < hb[y]; });
  double kept2 = 0;
  for (int64_t k = 0; k < chi; ++k) kept2 += hs[k] * hs[k];
  const double scale = (renorm && kept2 > 0) ? 1.0 / sqrt(kept2) : 1.0;
  std::vector<KeptIdx> hk(chi);
  for (int64_t k = 0; k < chi; ++k) {
    const int e = order[k];
    const Blk& B = bl[hb[e]];
    KeptIdx& K = hk[k];
    K.voff = B.goff;
    K.vld = B.g;
    K.xoff = B.xoff;
    K.xld = (side == TNT_SVD_LEFT) ? B.nq : B.k;
    K.roff = B.roff;
    K.nr = B.mq;
    K.coff = B.coff;
    K.nc = B.nq;
    K.loc = hl[e];
    K.blk = hb[e];
    h_S[k] = hs[e] * scale;
    h_bq[k] = B.q;
  }
  KeptIdx* d_kept = (KeptIdx*)ws_alloc(c, ws_round(sizeof(KeptIdx) * chi));
  if (!d_kept) return set_err(c, TNT_E_ALLOC, "scratch exhausted (svd kept)");
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_kept, hk.data(), sizeof(KeptIdx) * chi, cudaMemcpyHostToDevice, st));
  TNT_TRY(zfill(c, U, m * chi, zmk(0, 0)));
  TNT_TRY(zfill(c, X, chi * n, zmk(0, 0)));
  int64_t mx = std::max(m, n);
  dim3 gs((unsigned)std::min<int64_t>((mx + 255) / 256, 16), (unsigned)chi);
  k_scatter<<<gs, 256, 0, st>>>(Vp, Xp, d_kept, d_rows, d_cols, d_unscale, side, scale, chi, n, U, X);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  TNT_CUDA_TRY(c, cudaStreamSynchronize(st));  // host tables (hk) die at return
  res->chi = chi;
  res->err = sel.err;
  res->disc = sel.disc;
  res->norm2 = sel.norm2;
  res->n_blocks = nb;
  res->tie_at_cut = sel.tie;
  return TNT_OK;
}

}  // namespace tnt

extern "C" int tnt_autoblock_components(int64_t m, int64_t n, const uint32_t* h_mask,
                                        int64_t* h_row_q, int64_t* h_col_q, int64_t* h_count) {
  if (m < 1 || n < 1 || !h_mask || !h_row_q || !h_col_q || !h_count) return TNT_E_INVALID;
  *h_count = tnt::autoblock_components(m, n, h_mask, h_row_q, h_col_q);
  return TNT_OK;
}
