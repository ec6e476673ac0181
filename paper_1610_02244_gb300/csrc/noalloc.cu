// H_eff.theta for callers that cannot allocate device memory.
//
// Some users of this library must not call cudaMalloc at all: a plug-in loaded into a host
// application that owns every byte of device memory (through its own pool allocator, or a
// budget fixed at start-up), and a process sharing its GPU with another framework that has
// reserved the rest, where any new allocation would fail or evict the other's memory.
// tnt_heff_apply_noalloc serves them.  It is the FP64 path of tnt_heff_apply with every
// intermediate placed in one file-scope device array of NOALLOC_BYTES instead of the
// context's scratch: the dense two-site operator W12 = W1.W2 (built on the device by one
// small kernel, so the call needs no host copy and no stream synchronisation), T1 = L.theta
// and T3 = W12.T1.  Every GPU that loads this library holds that array until the process
// exits.
//
// Host code sees only a host-side stand-in for the array's name, not a device address; a
// kernel handed the stand-in would fault or, where the GPU can reach host memory, silently
// use the wrong memory.  So the device address is looked up with cudaGetSymbolAddress once
// per device, on the first call made on that device (with that device current), and
// cached.  That lookup can initialise the module, so the first call on each device should
// come before any stream capture.
//
// All calls share the one array and it keeps the last call's contents.  Calls that overlap
// on the GPU (on different streams, or from different host threads using the same device)
// race on it.  Nothing in it needs to start at zero: each call overwrites W12 and both
// intermediates in full before reading them.
#include <atomic>

#include "heff_plan.cuh"

namespace tnt {

namespace {
constexpr size_t NOALLOC_BYTES = (size_t)16 << 20;   // 16 MiB per device
constexpr size_t NOALLOC_W12 = (size_t)1 << 20;      // dense W12 (<= 256 x 256): first 1 MiB
constexpr int NOALLOC_MAX_DEVICES = 64;
constexpr int64_t NOALLOC_LEG = 256;                  // d^2 D <= 256
// largest chl * D * d * d * chr: T1 and T3 share what W12 leaves
constexpr int64_t NOALLOC_MAX_T = (int64_t)((NOALLOC_BYTES - NOALLOC_W12) / 2 / sizeof(z));

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::atomic<void*> g_scratch_addr[NOALLOC_MAX_DEVICES];

int scratch_for_device(Ctx* c, unsigned char** out) {
  if (c->device < 0 || c->device >= NOALLOC_MAX_DEVICES)
    return set_err(c, TNT_E_UNSUPPORTED, "device ordinal %d beyond %d", c->device, NOALLOC_MAX_DEVICES);
  void* p = g_scratch_addr[c->device].load();
  if (!p) {
    TNT_CUDA_TRY(c, cudaSetDevice(c->device));
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_err(c, TNT_E_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                     cudaGetErrorString(e));
    g_scratch_addr[c->device].store(p);
  }
  *out = (unsigned char*)p;
  return TNT_OK;
}

// W12[i][j] = sum_w1 W1[w,w1,s1',s1] W2[w1,w2,s2',s2], i = (s1' s2' w2), j = (w s1 s2)
__global__ void k_noalloc_w12(const z* __restrict__ W1, const z* __restrict__ W2, int64_t d,
                              int64_t D, z* __restrict__ W12) {
  const int64_t nI = d * d * D, nJ = D * d * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nI * nJ;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / nJ, j = e % nJ;
    const int64_t w2 = i % D, s2o = (i / D) % d, s1o = i / (D * d);
    const int64_t s2 = j % d, s1 = (j / d) % d, w = j / (d * d);
    z acc = zmk(0, 0);
    for (int64_t w1 = 0; w1 < D; ++w1)
      zfma(acc, W1[((w * D + w1) * d + s1o) * d + s1], W2[((w1 * D + w2) * d + s2o) * d + s2]);
    W12[e] = acc;
  }
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
  if (d > NOALLOC_LEG || D > NOALLOC_LEG || d * d * D > NOALLOC_LEG)
    return set_err(c, TNT_E_UNSUPPORTED, "d^2 D = %lld exceeds %lld", (long long)(d * d * D),
                   (long long)NOALLOC_LEG);
  // each factor is checked before the product is formed, so the product cannot wrap
  if (chl > NOALLOC_MAX_T || chr > NOALLOC_MAX_T || chl * d * d * D > NOALLOC_MAX_T ||
      chl * d * d * D * chr > NOALLOC_MAX_T)
    return set_err(c, TNT_E_UNSUPPORTED,
                   "tnt_heff_apply_noalloc: chl*D*d*d*chr = %lld x %lld x %lld exceeds the %lld "
                   "entries its fixed %zu bytes of scratch hold (use tnt_heff_apply)",
                   (long long)chl, (long long)(D * d * d), (long long)chr,
                   (long long)NOALLOC_MAX_T, NOALLOC_BYTES);
  const int64_t t = chl * D * d * d * chr;
  unsigned char* base = nullptr;
  TNT_TRY(scratch_for_device(c, &base));
  OzOff fma_only(c);  // the tensor-core FP64 GEMM grows a buffer: FP64 FMA here
  cudaStream_t st = c->stream;
  const int64_t nI = d * d * D, nJ = D * d * d;
  z* W12 = (z*)base;
  z* T1 = (z*)(base + NOALLOC_W12);
  z* T3 = T1 + t;
  k_noalloc_w12<<<(unsigned)((nI * nJ + 255) / 256), 256, 0, st>>>((const z*)d_W1, (const z*)d_W2,
                                                                  d, D, W12);
  c->launches++;
  TNT_CHECK_LAUNCH(c);
  // T1[(a' w)][(s1 s2 b)] = sum_a L[(a' w)][a] theta[a][(s1 s2 b)]
  ZGemm g1{};
  g1.M = chl * D; g1.N = d * d * chr; g1.K = chl;
  g1.A = (const z*)d_L; g1.a_rs = chl; g1.a_cs = 1;
  g1.B = (const z*)d_theta; g1.b_rs = d * d * chr; g1.b_cs = 1;
  g1.C = T1; g1.c_rs = d * d * chr;
  g1.alpha = zmk(1, 0); g1.beta = zmk(0, 0); g1.batch = 1;
  TNT_TRY(zgemm(c, g1));
  // for each a': T3[a'][(s1' s2' w2)][b] = sum_{(w s1 s2)} W12[(s1' s2' w2)][(w s1 s2)] T1[a'][(w s1 s2)][b]
  ZGemm g2{};
  g2.M = nI; g2.N = chr; g2.K = nJ;
  g2.A = W12; g2.a_rs = nJ; g2.a_cs = 1; g2.a_bs = 0;
  g2.B = T1; g2.b_rs = chr; g2.b_cs = 1; g2.b_bs = nJ * chr;
  g2.C = T3; g2.c_rs = chr; g2.c_bs = nI * chr;
  g2.alpha = zmk(1, 0); g2.beta = zmk(0, 0); g2.batch = chl;
  TNT_TRY(zgemm(c, g2));
  // y[(a' s1' s2')][b'] = sum_{(w2 b)} T3[(a' s1' s2')][(w2 b)] R[b'][(w2 b)]
  ZGemm g4{};
  g4.M = chl * d * d; g4.N = chr; g4.K = D * chr;
  g4.A = T3; g4.a_rs = D * chr; g4.a_cs = 1;
  g4.B = (const z*)d_R; g4.b_rs = 1; g4.b_cs = D * chr;
  g4.C = (z*)d_y; g4.c_rs = chr;
  g4.alpha = zmk(1, 0); g4.beta = zmk(0, 0); g4.batch = 1;
  return zgemm(c, g4);
}
