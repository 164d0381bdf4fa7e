// Allocation-free density + smoothing-length solve for one small box.
//
// Some callers cannot call cudaMalloc: code that runs while a framework
// owns all device memory (a custom-call or plugin interface that hands in
// only preplanned buffers), code on a real-time or signal-driven path where
// an allocation may block or fail, and library users that must not grow
// the device footprint after start-up.  sph_density_small_noalloc serves
// them: it allocates nothing.  It is a variant of the smoothing-length
// update of the main path whose per-particle solver scratch (the FP64
// bracket, the flags, the running sums) lives in the file-scope device
// array below instead of context-owned buffers, with the neighbour sums
// taken by direct summation over the whole (small) box instead of the cell
// decomposition.  The caller still passes every input and output.
//
// The array holds SPH_NOALLOC_MAX_N particles (about 0.6 MB) and every GPU
// that loads the library keeps it until the process exits.  All calls on a
// device share it, so calls that overlap on the GPU (two streams, two
// host threads) race; it keeps the last call's contents, and each call
// clears what must start at zero.
#include <cmath>

#include "internal.cuh"

namespace {

constexpr int NA_MAX = SPH_NOALLOC_MAX_N;
constexpr int NA_TPB = 128;
constexpr float NA_SIGMA = 2.546479089470325f;  // 8/pi

struct NoallocScratch {
  double lo[NA_MAX];
  double hi[NA_MAX];
  float h[NA_MAX];
  float nngb[NA_MAX];
  float dnngb[NA_MAX];
  float rho[NA_MAX];
  int flag[NA_MAX];
  int nactive;
  int nlimit;
};

static __device__ __align__(256) NoallocScratch g_na_scratch;

// In host code g_na_scratch names a host-side stand-in, not a device
// address: na_scratch() looks the device address up for the current device.

enum : int { NA_ACTIVE = 1, NA_HI_VALID = 2 };

__global__ void k_na_init(int n, const float* h_guess, float h0, float hl, NoallocScratch* S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    S->nactive = 0;
    S->nlimit = 0;
  }
  if (i >= n) return;
  float v = h_guess ? h_guess[i] : h0;
  if (!(v > 0.f) || v > hl) v = hl;
  S->h[i] = v;
  S->lo[i] = 0.0;
  S->hi[i] = (double)hl;
  S->flag[i] = NA_ACTIVE;
}

// N_i, dN_i/dh and rho_i at the current h by direct summation over every
// particle (minimum image; valid while h <= box/2)
__global__ void k_na_density(int n, const double* pos, double box, const float* m,
                             NoallocScratch* S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !(S->flag[i] & NA_ACTIVE)) return;
  const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
  const float h = S->h[i];
  const float hinv = 1.0f / h;
  float s0 = 0.f, s2 = 0.f, s3 = 0.f;
  for (int j = 0; j < n; ++j) {
    double dxd = xi - pos[3 * j], dyd = yi - pos[3 * j + 1], dzd = zi - pos[3 * j + 2];
    dxd -= box * rint(dxd / box);
    dyd -= box * rint(dyd / box);
    dzd -= box * rint(dzd / box);
    float dx = (float)dxd, dy = (float)dyd, dz = (float)dzd;
    float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    float q = sqrtf(r2) * hinv;
    float a = fmaxf(1.f - q, 0.f), b = fmaxf(0.5f - q, 0.f);
    float a2 = a * a, b2 = b * b;
    float wh = fmaf(-4.f * b2, b, a2 * a);  // w/2
    float d6 = fmaf(4.f, b2, -a2);          // w'/6
    s0 = fmaf(m[j], wh, s0);
    s2 += wh;
    s3 = fmaf(q, d6, s3);
  }
  S->rho[i] = 2.f * NA_SIGMA * hinv * hinv * hinv * s0;
  S->nngb[i] = (64.f / 3.f) * s2;
  S->dnngb[i] = -64.f * hinv * s3;
}

// Newton step on N_i(h) - n_ngb inside the FP64 bracket (same rule as the
// cell-based solve; the limit is box/2 instead of a cell edge)
__global__ void k_na_update(int n, float n_ngb, float tol, float hl, NoallocScratch* S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int fl = S->flag[i];
  if (!(fl & NA_ACTIVE)) return;
  double hd = (double)S->h[i];
  double f = (double)S->nngb[i] - (double)n_ngb;
  if (fabs(f) <= (double)tol * (double)n_ngb) {
    S->flag[i] = fl & ~NA_ACTIVE;
    return;
  }
  double L = S->lo[i], H = S->hi[i];
  if (f < 0) {
    L = hd;
    if (hd >= (double)hl) {
      S->flag[i] = 0;
      atomicAdd(&S->nlimit, 1);
      return;
    }
  } else {
    H = hd;
    fl |= NA_HI_VALID;
  }
  double dN = (double)S->dnngb[i];
  double hn = dN > 0 ? hd - f / dN : -1.0;
  if (fl & NA_HI_VALID) {
    if (!(hn > L && hn < H)) hn = 0.5 * (L + H);
    if (H - L <= 2.4e-7 * hd) {
      S->lo[i] = L;
      S->hi[i] = H;
      S->flag[i] = fl & ~NA_ACTIVE;
      return;
    }
  } else {
    if (!(hn > L)) hn = 2.0 * hd;
    hn = fmin(hn, (double)hl);
  }
  float hf = (float)hn;
  S->lo[i] = L;
  S->hi[i] = H;
  if (hf == S->h[i]) {
    S->flag[i] = fl & ~NA_ACTIVE;
    return;
  }
  S->h[i] = hf;
  S->flag[i] = fl;
  atomicAdd(&S->nactive, 1);
}

__global__ void k_na_out(int n, const NoallocScratch* S, float* h_out, float* rho_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (h_out) h_out[i] = S->h[i];
  if (rho_out) rho_out[i] = S->rho[i];
}

// The device address of the scratch array on the current device.  It is
// looked up on every call (a cheap host-side lookup once the module is
// loaded; the first call on a device loads it), so no address is cached
// across a device reset.
int na_scratch(NoallocScratch** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
  if (e != cudaSuccess || !p) {
    fprintf(stderr, "sphgb: cudaGetSymbolAddress of the no-alloc scratch failed: %s\n",
            cudaGetErrorString(e));
    return SPH_ERR_CUDA;
  }
  *out = reinterpret_cast<NoallocScratch*>(p);
  return SPH_OK;
}

}  // namespace

extern "C" int sph_density_small_noalloc(int32_t n, const double* pos, double box, const float* m,
                                         const float* h_guess, float n_ngb, int32_t max_iter,
                                         float* h_out, float* rho_out, int32_t* iters,
                                         void* stream) {
  if (n > NA_MAX) {
    fprintf(stderr, "sphgb: sph_density_small_noalloc: n = %d exceeds SPH_NOALLOC_MAX_N = %d\n", n,
            NA_MAX);
    return SPH_ERR_INVALID_ARG;
  }
  if (n <= 0 || !pos || !m || !(box > 0) || !(n_ngb > 32.f / 3.f) || max_iter < 1 ||
      (!h_out && !rho_out))
    return SPH_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  NoallocScratch* S = nullptr;
  SPH_TRY(na_scratch(&S));
  const float hl = (float)(0.5 * box);
  // default guess: the h holding n_ngb particles at the box's mean density
  const float h0 = (float)fmin(cbrt(3.0 * n_ngb * box * box * box / (4.0 * M_PI * n)), 0.25 * box);
  const int grid = div_up(n, NA_TPB);
  { k_na_init<<<grid, NA_TPB, 0, s>>>(n, h_guess, h0, hl, S); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  const float tol = 1.0f / 524288.0f;  // 2^-19, as the cell-based solve
  int it = 0, host_active = 1;
  for (; it < max_iter; ++it) {
    { k_na_density<<<grid, NA_TPB, 0, s>>>(n, pos, box, m, S); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    SPH_CUDA(cudaMemsetAsync(&S->nactive, 0, sizeof(int), s));
    { k_na_update<<<grid, NA_TPB, 0, s>>>(n, n_ngb, tol, hl, S); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    SPH_CUDA(cudaMemcpyAsync(&host_active, &S->nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    if (host_active == 0) {
      ++it;
      break;
    }
  }
  if (host_active) {
    // out of iterations: the last update moved h of the particles still
    // iterating, so evaluate rho once more at that h (the outputs then
    // belong together even though the call reports H_NOT_CONVERGED)
    { k_na_density<<<grid, NA_TPB, 0, s>>>(n, pos, box, m, S); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  int host_limit = 0;
  SPH_CUDA(cudaMemcpyAsync(&host_limit, &S->nlimit, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPH_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  { k_na_out<<<grid, NA_TPB, 0, s>>>(n, S, h_out, rho_out); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  if (host_limit) return SPH_ERR_CELL_LIMIT;
  if (host_active) return SPH_ERR_H_NOT_CONVERGED;
  return SPH_OK;
}
