// H_eff.theta for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running while a CUDA stream is being
// captured into a graph, plug-ins living under a host application's own allocator or a
// fixed memory budget, and processes that must not grow their device footprint after
// start-up.  tnt_heff_apply_noalloc serves them: it is the FP64 path of tnt_heff_apply,
// with the two intermediates T1 = L.theta and T3 = W.W.T1 and the small operator tables
// placed in a file-scope device array of NOALLOC_BYTES instead of the context's scratch.
// Every GPU that loads this library holds that array until the process exits.
//
// Host code sees only a host-side stand-in for the array's name; the device address is
// looked up once per device with cudaGetSymbolAddress, on the first call made on that
// device (with the device current), and cached.  Because that lookup can initialise the
// module, the first call on each device should come before any stream capture.
//
// All calls share the one array and it keeps the last call's contents; calls that
// overlap on the GPU (different streams, or different host threads) race on it.  Nothing
// in it needs to start at zero: each call overwrites the tables and both intermediates in
// full before reading them.
#include <algorithm>

#include "heff_plan.cuh"

namespace tnt {

namespace {
constexpr size_t NOALLOC_BYTES = (size_t)16 << 20;   // 16 MiB per device
constexpr size_t NOALLOC_TABLES = (size_t)64 << 10;  // operator tables: first 64 KiB
constexpr int NOALLOC_MAX_DEVICES = 64;
constexpr int NOALLOC_LEG = 256;                      // d^2 D <= 256
constexpr int NOALLOC_NNZ = 2048;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

void* g_scratch_addr[NOALLOC_MAX_DEVICES] = {nullptr};

// host staging for the operator tables (static: no host allocation per call)
struct Staging {
  z W1[NOALLOC_LEG * 16], W2[NOALLOC_LEG * 16];  // D^2 d^2 <= 16 * 256
  z w12[NOALLOC_LEG * NOALLOC_LEG];
  int row[NOALLOC_LEG + 1];
  int col[NOALLOC_NNZ];
  z val[NOALLOC_NNZ];
  int64_t in_off[NOALLOC_LEG], out_off[NOALLOC_LEG];
};
Staging g_stage;

int scratch_for_device(Ctx* c, unsigned char** out) {
  if (c->device < 0 || c->device >= NOALLOC_MAX_DEVICES)
    return set_err(c, TNT_E_UNSUPPORTED, "device ordinal %d beyond %d", c->device, NOALLOC_MAX_DEVICES);
  if (!g_scratch_addr[c->device]) {
    TNT_CUDA_TRY(c, cudaSetDevice(c->device));
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_err(c, TNT_E_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                     cudaGetErrorString(e));
    g_scratch_addr[c->device] = p;
  }
  *out = (unsigned char*)g_scratch_addr[c->device];
  return TNT_OK;
}
}  // namespace

}  // namespace tnt

using namespace tnt;

extern "C" int tnt_heff_apply_noalloc(tnt_ctx* ctx, const tnt_cplx* d_L, const tnt_cplx* d_W1,
                                      const tnt_cplx* d_W2, const tnt_cplx* d_R,
                                      const tnt_cplx* d_theta, int64_t chl, int64_t d,
                                      int64_t D, int64_t chr, tnt_cplx* d_y) {
  if (!ctx) return TNT_E_INVALID;
  Ctx* c = &ctx->c;
  if (!d_L || !d_W1 || !d_W2 || !d_R || !d_theta || !d_y)
    return set_err(c, TNT_E_INVALID, "null pointer");
  if (d_y == d_theta) return set_err(c, TNT_E_INVALID, "d_y aliases d_theta");
  if (chl <= 0 || d <= 0 || D <= 0 || chr <= 0) return set_err(c, TNT_E_INVALID, "non-positive dimension");
  if (d * d * D > NOALLOC_LEG || D * D * d * d > NOALLOC_LEG * 16)
    return set_err(c, TNT_E_UNSUPPORTED, "d^2 D = %lld exceeds %d (or D^2 d^2 exceeds %d)",
                   (long long)(d * d * D), NOALLOC_LEG, NOALLOC_LEG * 16);
  const size_t t = (size_t)chl * D * d * d * chr;
  const size_t need = NOALLOC_TABLES + 2 * ws_round(sizeof(z) * t);
  if (need > NOALLOC_BYTES)
    return set_err(c, TNT_E_UNSUPPORTED,
                   "tnt_heff_apply_noalloc: chl*D*d*d*chr = %zu needs %zu bytes of scratch, more "
                   "than its fixed %zu bytes (use tnt_heff_apply)", t, need, NOALLOC_BYTES);
  unsigned char* base = nullptr;
  TNT_TRY(scratch_for_device(c, &base));
  OzOff fma_only(c);  // the tensor-core FP64 GEMM grows a buffer: FP64 FMA here
  Staging& S = g_stage;
  const size_t nW = (size_t)(D * D * d * d);
  TNT_TRY(read_small(c, d_W1, S.W1, nW * sizeof(z)));
  TNT_TRY(read_small(c, d_W2, S.W2, nW * sizeof(z)));
  // W12[(s1' s2' w2), (w s1 s2)] = sum_w1 W1[w,w1,s1',s1] W2[w1,w2,s2',s2], as CSR
  const int nI = (int)(d * d * D), nJ = (int)(D * d * d);
  int nnz = 0;
  S.row[0] = 0;
  for (int64_t s1o = 0; s1o < d; ++s1o)
    for (int64_t s2o = 0; s2o < d; ++s2o)
      for (int64_t w2 = 0; w2 < D; ++w2) {
        const int64_t i = (s1o * d + s2o) * D + w2;
        for (int64_t w = 0; w < D; ++w)
          for (int64_t s1 = 0; s1 < d; ++s1)
            for (int64_t s2 = 0; s2 < d; ++s2) {
              z acc = zmk(0, 0);
              for (int64_t w1 = 0; w1 < D; ++w1)
                zfma(acc, S.W1[((w * D + w1) * d + s1o) * d + s1],
                     S.W2[((w1 * D + w2) * d + s2o) * d + s2]);
              if (acc.x != 0.0 || acc.y != 0.0) {
                if (nnz >= NOALLOC_NNZ)
                  return set_err(c, TNT_E_UNSUPPORTED, "operator has more than %d nonzeros", NOALLOC_NNZ);
                S.col[nnz] = (int)((w * d + s1) * d + s2);
                S.val[nnz] = acc;
                ++nnz;
              }
            }
        S.row[i + 1] = nnz;
      }
  for (int j = 0; j < nJ; ++j) S.in_off[j] = (int64_t)j * chr;
  for (int i = 0; i < nI; ++i) S.out_off[i] = (int64_t)i * chr;
  // tables into the first 64 KiB of the static array
  unsigned char* tb = base;
  int* d_row = (int*)tb;
  int* d_col = (int*)(tb + 2048);
  z* d_val = (z*)(tb + 2048 + 4 * NOALLOC_NNZ);
  int64_t* d_in = (int64_t*)(tb + 2048 + 4 * NOALLOC_NNZ + 16 * NOALLOC_NNZ);
  int64_t* d_out = d_in + NOALLOC_LEG;
  cudaStream_t st = c->stream;
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_row, S.row, sizeof(int) * (nI + 1), cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_col, S.col, sizeof(int) * std::max(nnz, 1), cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_val, S.val, sizeof(z) * std::max(nnz, 1), cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_in, S.in_off, sizeof(int64_t) * nJ, cudaMemcpyHostToDevice, st));
  TNT_CUDA_TRY(c, cudaMemcpyAsync(d_out, S.out_off, sizeof(int64_t) * nI, cudaMemcpyHostToDevice, st));
  // the staging buffers are reused by the next call: wait for the copies
  TNT_CUDA_TRY(c, cudaStreamSynchronize(st));
  z* T1 = (z*)(base + NOALLOC_TABLES);
  z* T3 = (z*)(base + NOALLOC_TABLES + ws_round(sizeof(z) * t));
  // T1[(a' w)][(s1 s2 b)] = sum_a L[(a' w)][a] theta[a][(s1 s2 b)]
  ZGemm g1{};
  g1.M = chl * D; g1.N = d * d * chr; g1.K = chl;
  g1.A = (const z*)d_L; g1.a_rs = chl; g1.a_cs = 1;
  g1.B = (const z*)d_theta; g1.b_rs = d * d * chr; g1.b_cs = 1;
  g1.C = T1; g1.c_rs = d * d * chr;
  g1.alpha = zmk(1, 0); g1.beta = zmk(0, 0); g1.batch = 1;
  TNT_TRY(zgemm(c, g1));
  // T3 = W12 (x) T1 on the (w s1 s2) legs
  OpApply a{};
  a.in = T1; a.out = T3;
  a.nI = nI; a.nJ = nJ; a.nnz = nnz;
  a.row_ptr = d_row; a.col = d_col; a.val = d_val; a.in_off = d_in; a.out_off = d_out;
  a.B0 = chl; a.B1 = 1; a.B2 = chr;
  a.is0 = D * d * d * chr; a.os0 = d * d * D * chr;
  a.is2 = a.os2 = 1;
  TNT_TRY(op_apply(c, a));
  // y[(a' s1' s2')][b'] = sum_{(w2 b)} T3[(a' s1' s2')][(w2 b)] R[b'][(w2 b)]
  ZGemm g4{};
  g4.M = chl * d * d; g4.N = chr; g4.K = D * chr;
  g4.A = T3; g4.a_rs = D * chr; g4.a_cs = 1;
  g4.B = (const z*)d_R; g4.b_rs = 1; g4.b_cs = D * chr;
  g4.C = (z*)d_y; g4.c_rs = chr;
  g4.alpha = zmk(1, 0); g4.beta = zmk(0, 0); g4.batch = 1;
  return zgemm(c, g4);
}
