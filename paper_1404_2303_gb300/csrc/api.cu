// C ABI entry points (include/sphgb.h) and the per-particle kernels around
// the sweeps: gathers into cell order, the smoothing-length update of
// Eq. (nneigh), the ghost step, and scatters back to the caller's order.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace {

constexpr int TPB = 256;
constexpr float SIGMA = 2.546479089470325f;  // 8/pi

enum : int { HF_ACTIVE = 1, HF_HI_VALID = 2, HF_LIMIT = 4, HF_LO_VALID = 8,
              HF_SIDE = 16,     // the last evaluation moved the lower end
              HF_RUN1 = 32,     // ... and so did the one before (one-sided run, 2 bits)
              HF_RUNMASK = 96 };

__global__ void k_fill_mass(long long n, const int* perm, const float* m, float4* pos4) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s < n) pos4[s].w = m[perm[s]];
}

__global__ void k_gather(long long n, const int* perm, const float* in, float* out) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s < n) out[s] = in[perm[s]];
}

__global__ void k_scatter(long long n, const int* perm, const float* in, float* out) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s < n) out[perm[s]] = in[s];
}

__global__ void k_scatter_z(long long n, const int* perm, const float4* in, float* out) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s < n) out[perm[s]] = in[s].z;
}

__global__ void k_scatter_i(long long n, const int* perm, const int* in, int* out) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s < n) out[perm[s]] = in[s];
}

__global__ void k_check_h(long long n, const float* h, const float* hlim, float pad, int* status) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  float v = h[s];
  if (!(v > 0.f) || v > hlim[s] - pad) atomicOr(status, ST_CELL_LIMIT);
}

// ---- smoothing-length solve (Eq. (nneigh)): Newton steps on
// ln N(ln h) = ln n_ngb (the paper's Newton iteration with dN/dh computed
// alongside the sums, taken in log-log form so that it lands on the root in
// one step when N grows like h^3, with the Halley correction from d2N/dh2),
// safeguarded by an FP64 bracket [lo, hi].  Where the local step leaves the
// bracket (N can steepen abruptly: a dense group of neighbours entering the
// kernel support at once contributes (1 - r/h)^3 terms that the derivatives
// at the current h do not see), the step is the root of the cubic Hermite
// interpolant of g = ln(N / n_ngb) over the bracket, built from g and dg/dlnh
// recorded at both ends; bisection remains the last resort, so the bracket
// keeps shrinking.
struct HSolve {
  float* h;
  const float* hlim;
  const float* nngb;
  const float* dnngb;
  const float* d2nngb;
  double* lo;
  double* hi;
  float4* gb;      // g and dg/dlnh at the lower end (x, y) and the upper end (z, w)
  float* dxold;
  int* flag;
  float n_ngb, tol;
  float pad;       // the cell limit is hlim - pad (particles moved since the build)
  int* nactive;
  int* nlimit;
};

// mode 0: every particle starts; mode 1 (after a rebuild): only the particles
// whose root lay beyond their old cell limit restart, with the old limit as
// their evaluated lower end; the others keep their converged h and sums
__global__ void k_hsolve_init(long long n, HSolve S, int mode) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float hl = S.hlim[s] - S.pad;
  if (mode == 1) {
    const int fl = S.flag[s];
    if (!(fl & HF_LIMIT)) {
      S.flag[s] = 0;
      return;
    }
    S.hi[s] = (double)hl;
    S.dxold[s] = 1e30f;
    S.flag[s] = HF_ACTIVE | HF_LO_VALID;  // lo and gb.xy hold the old limit's values
    return;
  }
  float v = S.h[s];
  if (!(v > 0.f) || v > hl) v = hl;
  S.h[s] = v;
  S.lo[s] = 0.0;
  S.hi[s] = (double)hl;
  S.dxold[s] = 1e30f;
  S.flag[s] = HF_ACTIVE;
}

// root in (0, 1) of the cubic Hermite interpolant with values p0 < 0 < p1 and
// slopes m0, m1 (per unit t) at t = 0 and t = 1: Newton steps kept inside a
// shrinking sub-bracket; -1 if no usable root
__device__ double hermite_root(double p0, double m0, double p1, double m1) {
  double a = 0.0, b = 1.0;
  double t = p0 / (p0 - p1);  // the secant point
  for (int it = 0; it < 24; ++it) {
    const double t2 = t * t, t3 = t2 * t;
    const double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t, h01 = -2 * t3 + 3 * t2,
                 h11 = t3 - t2;
    const double c = h00 * p0 + h10 * m0 + h01 * p1 + h11 * m1;
    const double dc = (6 * t2 - 6 * t) * p0 + (3 * t2 - 4 * t + 1) * m0 + (-6 * t2 + 6 * t) * p1 +
                      (3 * t2 - 2 * t) * m1;
    if (c < 0) a = t; else b = t;
    if (fabs(c) < 1e-12) return t;
    double tn = dc > 0 ? t - c / dc : -1.0;
    if (!(tn > a && tn < b)) tn = 0.5 * (a + b);
    if (fabs(tn - t) < 1e-14) return tn;
    t = tn;
  }
  return (b - a) < 1e-6 ? 0.5 * (a + b) : -1.0;
}

// |ln(a / b)| for the step-size bookkeeping, in FP32 (the bracket ends and
// h are FP32 values held in FP64; FP64 transcendentals are slow here)
__device__ __forceinline__ float log_ratio(double a, double b) {
  return fabsf(log1pf((float)(a - b) / (float)b));
}

__global__ void k_hsolve_update(long long n, HSolve S) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  int fl = S.flag[s];
  if (!(fl & HF_ACTIVE)) return;
  const double hd = (double)S.h[s];
  const float Nv = S.nngb[s];
  const double f = (double)Nv - (double)S.n_ngb;
  if (fabs(f) <= (double)S.tol * (double)S.n_ngb) {
    S.flag[s] = fl & ~HF_ACTIVE;
    return;
  }
  double L = S.lo[s], H = S.hi[s];
  float4 gb = S.gb[s];
  const double hl = (double)(S.hlim[s] - S.pad);
  // g(x) = ln N - ln n_ngb and g'(x) = h N'/N in x = ln h
  const float slope = (S.dnngb[s] > 0.f && Nv > 0.f) ? (float)(hd * (double)S.dnngb[s] / (double)Nv) : 0.f;
  const float g = __logf(Nv) - __logf(S.n_ngb);
  // runs of evaluations on one side of the root (counted up to 3): an
  // interpolation that keeps landing on the same side is replaced by
  // bisection, which halves the bracket from that side
  const int side = f < 0 ? HF_SIDE : 0;
  int run = (fl & HF_RUNMASK) / HF_RUN1;
  run = ((fl & HF_SIDE) == side) ? min(run + 1, 3) : 0;
  fl = (fl & ~(HF_SIDE | HF_RUNMASK)) | side | (run * HF_RUN1);
  if (f < 0) {
    L = hd;
    gb.x = g;
    gb.y = slope;
    fl |= HF_LO_VALID;
    if (hd >= hl) {  // the root lies beyond what this decomposition covers
      S.lo[s] = L;
      S.gb[s] = gb;
      S.flag[s] = HF_LIMIT | HF_LO_VALID;
      atomicAdd(S.nlimit, 1);
      return;
    }
  } else {
    H = hd;
    gb.z = g;
    gb.w = slope;
    fl |= HF_HI_VALID;
  }
  // Halley step ln(h / h_new) from the current point, with
  // g''(x) = g' + h^2 N''/N - g'^2 (the Newton step g/g' where the
  // correction is not well conditioned)
  float dx = slope > 1e-3f ? g / slope : 0.f;
  if (slope > 1e-3f) {
    const float hf0 = (float)hd;
    const float curv = slope + hf0 * hf0 * S.d2nngb[s] / Nv - slope * slope;
    const float den = 2.f * slope * slope - g * curv;
    if (den > slope * slope) dx = 2.f * g * slope / den;
  }
  const float dxprev = S.dxold[s];
  double hn;
  float step;
  if (fl & HF_HI_VALID) {
    if (H - L <= 2.4e-7 * hd) {  // bracket below FP32 resolution
      S.lo[s] = L;
      S.hi[s] = H;
      S.gb[s] = gb;
      S.flag[s] = fl & ~HF_ACTIVE;
      return;
    }
    const double prop = slope > 1e-3f ? hd * (double)__expf(-dx) : -1.0;
    const bool out = !(prop > L && prop < H);
    // a step that is not at least twice shorter than the one before gives
    // way to the bracket (only once both of its ends are evaluated: without
    // a lower end the fallback would halve h)
    const bool slow = (fl & HF_LO_VALID) && fabsf(2.f * g) > fabsf(dxprev * slope);
    hn = -1.0;
    if (!(out || slow || slope <= 1e-3f)) {
      hn = prop;
    } else if ((fl & HF_LO_VALID) && L > 0 && gb.y > 0.f && gb.w > 0.f && run < 3) {
      // cubic Hermite interpolation of g over [ln L, ln H]: accurate to the
      // fourth order in the bracket width, so its root is taken even when it
      // lies far from the current end (no step-length test)
      // (increments relative to L kept exact: the bracket can be a few
      // FP32 ulps wide)
      const float x = (float)((H - L) / L);
      const double w = (double)log1pf(x);
      const double t = hermite_root((double)gb.x, (double)gb.y * w, (double)gb.z, (double)gb.w * w);
      if (t > 0.0 && t < 1.0) {
        const double q = L + L * (double)expm1f((float)(t * w));
        if (q > L && q < H) hn = q;
      }
    }
    if (!(hn > 0)) {  // bisection (geometric once L > 0)
      if (L > 0) {
        const float x = (float)((H - L) / L);
        hn = L + L * (double)(x / (sqrtf(1.f + x) + 1.f));
      } else {
        hn = 0.5 * (L + H);
      }
    }
    step = log_ratio(hn, hd);
  } else {
    // no upper end yet: Newton upwards, doubling when it has no slope, capped
    // at the cell limit (evaluated there once before declaring the limit)
    hn = slope > 1e-3f ? hd * (double)__expf(-dx) : 2.0 * hd;
    if (!(hn > L)) hn = 2.0 * hd;
    hn = fmin(hn, hl);
    step = log_ratio(hn, hd);
  }
  S.lo[s] = L;
  S.hi[s] = H;
  S.gb[s] = gb;
  S.dxold[s] = step;
  const float hf = (float)hn;
  if (hf == S.h[s] || step < 1e-7f) {  // no FP32-representable progress left
    S.flag[s] = fl & ~HF_ACTIVE;
    return;
  }
  S.h[s] = hf;
  S.flag[s] = fl;
  atomicAdd(S.nactive, 1);
}

// body end of the device-side h iteration: record this iteration's active
// count and continue while particles are still iterating (max_newton cap)
__global__ void k_loop_ctl(const int* nact, int* iter, int* hist, int maxit,
                           cudaGraphConditionalHandle hnd) {
  const int it = *iter, na = *nact;
  if (it < 32) hist[it] = na;
  *iter = it + 1;
  cudaGraphSetConditional(hnd, (na > 0 && it + 1 < maxit) ? 1u : 0u);
}

__global__ void k_block_active(int nblock, const int* b_first, const int* b_count, const int* flag,
                               int* act) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= nblock) return;
  int f = b_first[warp], c = b_count[warp];
  int any = 0;
  for (int k = lane; k < c; k += 32) any |= flag[f + k] & HF_ACTIVE;
  any = __any_sync(0xffffffffu, any);
  if (lane == 0) act[warp] = any;
}

// build guess of the next decomposition: the current h, and for particles
// whose root lies beyond their cell limit the larger of twice the limit and
// the h at which N would reach n_ngb if it grew like h^3 from its value at
// the limit (with a 25 % margin)
__global__ void k_rebuild_guess(long long n, const float* h, const float* hlim, const int* flag,
                                const float* nngb, float n_ngb, float* hg) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  if (flag[s] & HF_LIMIT) {
    const float hl = hlim[s], N = nngb[s];
    const float ext = N > 0.f ? 1.25f * cbrtf(n_ngb / N) : 2.f;
    hg[s] = hl * fmaxf(2.f, ext);
  } else {
    hg[s] = h[s];
  }
}

// ---- ghost step (text after Eq. (dudt)) and force-side per-particle data
__global__ void k_ghost(long long n, const int* perm, const float* h, const float4* pos4,
                        const float* rho, const float* drho, const float* u, const float* vel,
                        float gamma, float* omega, float* Avec, float* u_s, float4* vel4,
                        float4* fdat) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  int p = perm[s];
  float hv = h[s], r = rho[s];
  float om = 1.f + hv * drho[s] / (3.f * r);
  float uu = u[p];
  float P = (gamma - 1.f) * r * uu;
  float A = P / (om * r * r);
  float hi = 1.f / hv;
  float hi2 = hi * hi;
  float C = 6.f * SIGMA * A * hi2 * hi2;
  omega[s] = om;
  Avec[s] = A;
  u_s[s] = uu;
  float4 v = make_float4(0.f, 0.f, 0.f, hi);
  if (vel) {
    v.x = vel[3 * (long long)p];
    v.y = vel[3 * (long long)p + 1];
    v.z = vel[3 * (long long)p + 2];
  }
  vel4[s] = v;
  fdat[s] = make_float4(pos4[s].w * C, __fmul_rn(hv, hv), C, A);
}

__global__ void k_scatter_acc(long long n, const int* perm, const float4* acc4, float* acc,
                              float* dudt) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  int p = perm[s];
  float4 a = acc4[s];
  acc[3 * (long long)p] = a.x;
  acc[3 * (long long)p + 1] = a.y;
  acc[3 * (long long)p + 2] = a.z;
  if (dudt) dudt[p] = a.w;
}

__global__ void k_sum_i32(long long n, const int* v, unsigned long long* out) {
  __shared__ unsigned long long sm[TPB / 32];
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  unsigned long long x = s < n ? (unsigned long long)v[s] : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < TPB / 32; ++k) t += sm[k];
    atomicAdd(out, t);
  }
}

}  // namespace

// ===========================================================================
static cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

static int status_from_word(int w) {
  if (w & ST_BAD_INPUT) return SPH_ERR_INVALID_ARG;
  if (w & ST_CAPACITY) return SPH_ERR_CAPACITY;
  if (w & ST_TIMEOUT) return SPH_ERR_TIMEOUT;
  if (w & ST_CELL_LIMIT) return SPH_ERR_CELL_LIMIT;
  if (w & ST_NOT_CONVERGED) return SPH_ERR_H_NOT_CONVERGED;
  if (w & ST_BAD_INDEX) return SPH_ERR_CUDA;
  return SPH_OK;
}

static int read_status(sph_ctx* c, cudaStream_t s) {
  int w = 0;
  SPH_CUDA(cudaMemcpyAsync(&w, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPH_CUDA(cudaStreamSynchronize(s));
  if (w) SPH_CUDA(cudaMemsetAsync(c->status.p, 0, sizeof(int), s));
  return status_from_word(w);
}

static int ensure_state(sph_ctx* c) {
  const size_t n = (size_t)c->n;
  DBuf* f1[] = {&c->rho, &c->drho, &c->nngb, &c->dnngb, &c->d2nngb, &c->d2rho, &c->omega, &c->Avec, &c->u_s};
  for (DBuf* b : f1) SPH_TRY(dbuf_ensure(*b, 4 * n));
  SPH_TRY(dbuf_ensure(c->fdat, 16 * n));
  SPH_TRY(dbuf_ensure(c->vel4, 16 * n));
  SPH_TRY(dbuf_ensure(c->acc4, 16 * n));
  SPH_TRY(dbuf_ensure(c->cnt_i, 4 * n));
  SPH_TRY(dbuf_ensure(c->h_lo, 8 * n));
  SPH_TRY(dbuf_ensure(c->h_hi, 8 * n));
  SPH_TRY(dbuf_ensure(c->h_flag, 4 * n));
  SPH_TRY(dbuf_ensure(c->h_dx, 4 * n));
  SPH_TRY(dbuf_ensure(c->h_gb, 16 * n));
  SPH_TRY(dbuf_ensure(c->blk_active, 4 * (size_t)(c->nblock + 1)));
  SPH_TRY(dbuf_ensure(c->tmp_a, 64));
  return SPH_OK;
}

static HSolve hsolve_args(sph_ctx* c, int* nactive, int* nlimit) {
  HSolve S;
  S.h = c->h.as<float>();
  S.hlim = c->hlim.as<float>();
  S.nngb = c->nngb.as<float>();
  S.dnngb = c->dnngb.as<float>();
  S.d2nngb = c->d2nngb.as<float>();
  S.lo = c->h_lo.as<double>();
  S.hi = c->h_hi.as<double>();
  S.gb = c->h_gb.as<float4>();
  S.dxold = c->h_dx.as<float>();
  S.flag = c->h_flag.as<int>();
  S.n_ngb = c->prm.n_ngb;
  S.tol = c->prm.h_tol;
  S.pad = c->reuse_pad;
  S.nactive = nactive;
  S.nlimit = nlimit;
  return S;
}

static int count_total(sph_ctx* c, unsigned long long* out, cudaStream_t s) {
  unsigned long long* d = c->counters.as<unsigned long long>() + 1;
  SPH_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long), s));
  { k_sum_i32<<<div_up(c->n, TPB), TPB, 0, s>>>(c->n, c->cnt_i.as<int>(), d); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_CUDA(cudaMemcpyAsync(out, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  SPH_CUDA(cudaStreamSynchronize(s));
  return SPH_OK;
}

static void graph_release(sph_ctx* c) {
  if (c->g_exec) cudaGraphExecDestroy(c->g_exec);
  if (c->g_graph) cudaGraphDestroy(c->g_graph);
  c->g_exec = nullptr;
  c->g_graph = nullptr;
}

// One solve round as a CUDA graph: a WHILE conditional node whose body
// (active blocks, density sweep over them, h update, loop control) runs
// on the device until no particle is iterating or max_newton is reached;
// the host reads the counters once at the end.  The graph bakes in the
// decomposition's buffers, so it is captured again after every build.
static int solve_round_graph(sph_ctx* c, cudaStream_t s, int* host, int* iters, int hist0) {
  const long long n = c->n;
  int* ctl = c->solve_ctl.as<int>();  // [0] active [1] at limit [2] iteration [3..34] history
  if (!c->g_exec || c->g_gen != c->build_gen) {
    graph_release(c);
    cudaGraph_t g = nullptr;
    SPH_CUDA(cudaGraphCreate(&g, 0));
    c->g_graph = g;
    cudaGraphConditionalHandle hnd;
    SPH_CUDA(cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hnd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn;
    SPH_CUDA(cudaGraphAddNode(&cn, g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs = c->cap_stream;
    const long long before = launch_count();
    SPH_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    int r = SPH_OK;
    { k_block_active<<<div_up((long long)c->nblock * 32, TPB), TPB, 0, cs>>>(
        c->nblock, c->b_first.as<int>(), c->b_count.as<int>(), c->h_flag.as<int>(),
        c->blk_active.as<int>()); note_launch(); }
    if (r == SPH_OK) r = run_sweep(c, PH_DENSITY, 1, 0, cs);
    if (r == SPH_OK && cudaMemsetAsync(ctl, 0, sizeof(int), cs) != cudaSuccess) r = SPH_ERR_CUDA;
    { k_hsolve_update<<<div_up(n, TPB), TPB, 0, cs>>>(n, hsolve_args(c, ctl, ctl + 1)); note_launch(); }
    { k_loop_ctl<<<1, 1, 0, cs>>>(ctl, ctl + 2, ctl + 3, c->prm.max_newton, hnd); note_launch(); }
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &captured);
    c->g_body_kernels = launch_count() - before;  // captured, not executed
    note_launch_n(-c->g_body_kernels);
    if (r != SPH_OK) return r;
    SPH_CUDA(e);
    SPH_CUDA(cudaGraphInstantiate(&c->g_exec, g, 0));
    c->g_gen = c->build_gen;
  }
  SPH_CUDA(cudaMemsetAsync(ctl + 1, 0, 34 * sizeof(int), s));
  SPH_CUDA(cudaGraphLaunch(c->g_exec, s));
  int h_ctl[35];
  SPH_CUDA(cudaMemcpyAsync(h_ctl, ctl, sizeof(h_ctl), cudaMemcpyDeviceToHost, s));
  SPH_CUDA(cudaStreamSynchronize(s));
  host[0] = h_ctl[0];
  host[1] = h_ctl[1];
  *iters = h_ctl[2];
  note_launch_n(c->g_body_kernels * h_ctl[2]);  // body kernels the graph ran
  for (int k = 0; k < 32 && hist0 + k < 32; ++k) c->stats.newton_active[hist0 + k] = h_ctl[3 + k];
  return SPH_OK;
}

extern "C" {

void sph_default_params(sph_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->n_ngb = 48.0f;
  p->gamma = 5.0f / 3.0f;
  p->split_count = 300;
  p->split_frac = 0.875f;
  p->block_max = 64;
  p->max_newton = 64;
  p->max_rebuild = 4;
  p->kahan = 1;
  p->morton_bits = 16;
  p->h_tol = 1.0f / 524288.0f;  // 2^-19
  p->warps_per_cta = 8;
  p->ctas_per_sm = 0;
  p->h_est_mode = 1;
  p->h_est_factor = 1.5f;
  p->sweep_cap = 128;
  p->use_graph = 1;
  p->sweep_lists = 0x08;
  p->pair_list_cap = 256;
  p->list_cap = 4096;
  p->sorted_sweep = 1;
}

int sph_create(const sph_params* p, sph_ctx** out) {
  if (!out) return SPH_ERR_INVALID_ARG;
  *out = nullptr;
  sph_params q;
  if (p) q = *p; else sph_default_params(&q);
  if (!(q.n_ngb > 32.f / 3.f) || !(q.gamma > 1.f) || q.split_count < 1 || !(q.split_frac > 0.f) ||
      q.block_max < 32 || q.block_max > 256 || q.max_newton < 1 || q.max_rebuild < 0 ||
      q.morton_bits < 8 || q.morton_bits > 20 || !(q.h_tol > 0.f) || q.warps_per_cta < 1 ||
      q.warps_per_cta > 8 || q.ctas_per_sm < 0 || q.h_est_mode < 0 || q.h_est_mode > 1 ||
      !(q.h_est_factor > 0.f) || q.sweep_cap < 32 || q.sweep_cap > 1024 || (q.sweep_cap % 32) != 0 ||
      q.sweep_lists < 0 || q.sweep_lists > 0x1f || q.pair_list_cap < 0 || q.pair_list_cap > 4096 ||
      q.list_cap < 0 || q.list_cap > 4096 || q.sorted_sweep < 0 || q.sorted_sweep > 1)
    return SPH_ERR_INVALID_ARG;
  sph_ctx* c = new sph_ctx();
  c->prm = q;
  c->kbits = q.morton_bits;
  c->sweep_cap = q.sweep_cap;
  int r;
  if ((r = dbuf_ensure(c->status, 64)) != SPH_OK || (r = dbuf_ensure(c->counters, 64)) != SPH_OK ||
      (r = dbuf_ensure(c->queue, 64)) != SPH_OK) {
    sph_destroy(c);
    return r;
  }
  cudaMemset(c->status.p, 0, 64);
  cudaMemset(c->counters.p, 0, 64);
  if ((r = dbuf_ensure(c->solve_ctl, 64 * sizeof(int))) != SPH_OK ||
      cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      (r = set_dir_table(c)) != SPH_OK) {
    sph_destroy(c);
    return r != SPH_OK ? r : SPH_ERR_CUDA;
  }
  *out = c;
  return SPH_OK;
}

void sph_destroy(sph_ctx* c) {
  if (!c) return;
  DBuf* all[] = {&c->d_box_off, &c->d_box_L, &c->d_box_t, &c->d_top_base, &c->keys, &c->keys_alt,
                 &c->perm, &c->perm_alt, &c->xs, &c->pos4, &c->h, &c->hguess, &c->hlim, &c->pnode,
                 &c->n_first, &c->n_count, &c->n_parent, &c->n_child0, &c->n_top, &c->n_flags,
                 &c->n_need, &c->n_ijk, &c->n_box, &c->n_hmax, &c->n_hbuild, &c->n_hlim,
                 &c->n_sbase, &c->n_nblk, &c->n_blk0, &c->b_hmax, &c->t_cur, &c->t_next, &c->t_final_pair, &c->t_final_self, &c->t_cnt,
                 &c->t_cnt2, &c->t_off, &c->t_off2, &c->b_first, &c->b_count, &c->b_leaf,
                 &c->b_dtoff, &c->b_order, &c->b_cost, &c->dt_cj, &c->dt_code, &c->dt_shift,
                 &c->adj_off, &c->adj_list, &c->s_key, &c->s_idx, &c->rho, &c->drho, &c->nngb,
                 &c->dnngb, &c->d2nngb, &c->d2rho, &c->omega, &c->Avec, &c->fdat, &c->vel4, &c->u_s, &c->acc4,
                 &c->cnt_i, &c->h_lo, &c->h_hi, &c->h_dx, &c->h_gb, &c->h_flag, &c->blk_active, &c->adj4, &c->adj4b, &c->g_A,
                 &c->g_rho_s, &c->g_drho_s, &c->g_h_s, &c->g_u_s, &c->g_x4,
                 &c->prof_units, &c->solve_ctl, &c->status, &c->counters, &c->queue, &c->scan_tmp, &c->sort_tmp, &c->tmp_a,
                 &c->tmp_b, &c->tmp_c, &c->p_et, &c->nleaf_dev, &c->n_listed, &c->n_ex, &c->n_lo,
                 &c->n_hi, &c->b_lo, &c->b_hi, &c->fl_list, &c->fl_cnt, &c->fl_flag, &c->fl_blk,
                 &c->fl_over, &c->task_ctl, &c->tree_ctl, &c->visc4, &c->dt_s,
                 &c->b_nseg, &c->u_off, &c->b_part, &c->u_block, &c->u_seg, &c->u_e0, &c->u_e1,
                 &c->u_key, &c->part, &c->blk_done, &c->vv_acc, &c->vv_du, &c->vv_dt,
                 &c->vv_vp, &c->vv_up, &c->vv_h, &c->vv_tmp, &c->vv_red, &c->plan_max,
                 &c->u_act, &c->sl_list};
  for (DBuf* b : all) dbuf_free(*b);
  for (auto& e : c->ev_pending) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  graph_release(c);
  if (c->tree_host) cudaFreeHost(c->tree_host);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

int sph_build_batch(sph_ctx* c, int32_t nbox, const int64_t* offsets, const double* boxes,
                    const double* pos, const float* h_guess, void* stream) {
  if (!c || nbox < 1 || nbox > SPH_MAX_BOX || !offsets || !boxes || !pos)
    return SPH_ERR_INVALID_ARG;
  if (offsets[0] != 0) return SPH_ERR_INVALID_ARG;
  for (int b = 0; b < nbox; ++b)
    if (offsets[b + 1] <= offsets[b] || !(boxes[b] > 0)) return SPH_ERR_INVALID_ARG;
  long long n = offsets[nbox];
  if (n <= 0 || n >= (1ll << 31) / 16) return SPH_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  ++c->state_gen;
  if (c->reuse_pad != 0.f) ++c->build_gen;
  c->reuse_pad = 0.f;
  c->built = c->have_density = c->have_force = false;
  c->fl_valid = false;
  c->have_d2 = 0;
  c->n = n;
  c->nbox = nbox;
  c->box_off.assign(offsets, offsets + nbox + 1);
  c->box_L.assign(boxes, boxes + nbox);
  c->box_t.assign(nbox, 2);
  SPH_TRY(dbuf_ensure(c->d_box_off, sizeof(long long) * (nbox + 1)));
  SPH_TRY(dbuf_ensure(c->d_box_L, sizeof(double) * nbox));
  SPH_TRY(dbuf_ensure(c->d_box_t, sizeof(int) * nbox));
  SPH_TRY(dbuf_ensure(c->d_top_base, sizeof(int) * (nbox + 1)));
  SPH_CUDA(cudaMemcpyAsync(c->d_box_off.p, c->box_off.data(), sizeof(long long) * (nbox + 1),
                           cudaMemcpyHostToDevice, s));
  SPH_CUDA(cudaMemcpyAsync(c->d_box_L.p, c->box_L.data(), sizeof(double) * nbox,
                           cudaMemcpyHostToDevice, s));
  SPH_CUDA(cudaMemsetAsync(c->status.p, 0, sizeof(int), s));
  SPH_TRY(build_decomposition(c, pos, h_guess, s));
  SPH_TRY(ensure_state(c));
  int st = read_status(c, s);
  if (st != SPH_OK) return st;
  c->built = true;
  return SPH_OK;
}

int sph_build(sph_ctx* c, int64_t n, const double* pos, double box, const float* h_guess,
              void* stream) {
  int64_t off[2] = {0, n};
  return sph_build_batch(c, 1, off, &box, pos, h_guess, stream);
}

static int prep_mass(sph_ctx* c, const float* m, cudaStream_t s) {
  { k_fill_mass<<<div_up(c->n, TPB), TPB, 0, s>>>(c->n, c->perm.as<int>(), m, c->pos4.as<float4>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  return SPH_OK;
}

int sph_density_fixed_h(sph_ctx* c, const float* m, const float* h, float* rho, float* drho_dh,
                        float* nngb, float* dnngb_dh, int32_t* count, void* stream) {
  if (!c || !m || !h || !rho) return SPH_ERR_INVALID_ARG;
  if (!c->built) return SPH_ERR_NOT_BUILT;
  ++c->state_gen;
  cudaStream_t s = as_stream(stream);
  const long long n = c->n;
  SPH_TRY(prep_mass(c, m, s));
  { k_gather<<<div_up(n, TPB), TPB, 0, s>>>(n, c->perm.as<int>(), h, c->h.as<float>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  { k_check_h<<<div_up(n, TPB), TPB, 0, s>>>(n, c->h.as<float>(), c->hlim.as<float>(),
                                           c->reuse_pad, c->status.as<int>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(compute_node_hmax(c, s));
  SPH_TRY(run_sweep(c, PH_DENSITY, 0, count != nullptr, s));
  const int* perm = c->perm.as<int>();
  { k_scatter<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->rho.as<float>(), rho); note_launch(); }
  { if (drho_dh) k_scatter<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->drho.as<float>(), drho_dh); note_launch(); }
  { if (nngb) k_scatter<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->nngb.as<float>(), nngb); note_launch(); }
  { if (dnngb_dh) k_scatter<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->dnngb.as<float>(), dnngb_dh); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  c->have_density = true;
  c->have_force = false;
  c->fl_valid = false;
  c->have_d2 = 0;
  if (count) {
    { k_scatter_i<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->cnt_i.as<int>(), count); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    unsigned long long tot = 0;
    SPH_TRY(count_total(c, &tot, s));
    c->stats.density_interactions = (int64_t)tot;
    return read_status(c, s);
  }
  return SPH_OK;
}

int sph_density(sph_ctx* c, const float* m, float* h_out, float* rho, float* omega,
                int32_t* iters, void* stream) {
  if (!c || !m) return SPH_ERR_INVALID_ARG;
  if (!c->built) return SPH_ERR_NOT_BUILT;
  ++c->state_gen;
  cudaStream_t s = as_stream(stream);
  const long long n = c->n;
  SPH_TRY(prep_mass(c, m, s));
  int total_iters = 0, rebuilds = 0;
  int* nact = c->tmp_a.as<int>();
  int* nlim = nact + 1;
  for (int k = 0; k < 32; ++k) c->stats.newton_active[k] = 0;
  for (;;) {
    // the first round starts every particle; a round after a rebuild only
    // the particles whose root lay beyond their old cell limit
    { k_hsolve_init<<<div_up(n, TPB), TPB, 0, s>>>(n, hsolve_args(c, nact, nlim), rebuilds > 0 ? 1 : 0); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    int host[2] = {1, 0};
    int it = 0;
    SPH_CUDA(cudaMemsetAsync(c->blk_active.p, 0, 4 * (size_t)c->nblock, s));
    // nlim accumulates over the whole solve: a particle flagged at its cell
    // limit in any iteration leaves the active set and must trigger the rebuild
    SPH_CUDA(cudaMemsetAsync(nlim, 0, sizeof(int), s));
    // The work units were planned from the build's h.  Before each sweep of
    // the iteration the block costs are estimated again from the current h
    // of the particles still iterating, and the units re-planned when the
    // present plan would leave one unit far above its balanced share (the h
    // of particles next to dense clumps can grow tenfold over the first
    // iterations, and with it their candidate sets).  While the plan holds,
    // the rest of the round runs as one device-side graph.
    bool use_dev = c->prm.use_graph && !c->profile;
    bool replanned = false;
    // the first iteration of a fresh decomposition runs on the host, so that
    // the plan is checked against the h of the first Halley step
    const int min_host = rebuilds == 0 ? 1 : 0;
    for (; use_dev && it < c->prm.max_newton;) {
      bool changed = false;
      SPH_TRY(replan_units(c, 1, &changed, s));
      replanned = replanned || changed;
      if (!changed && !replanned && it >= min_host) break;  // a balanced plan: the graph takes the round
      SPH_TRY(ensure_state(c));
      { k_block_active<<<div_up((long long)c->nblock * 32, TPB), TPB, 0, s>>>(
          c->nblock, c->b_first.as<int>(), c->b_count.as<int>(), c->h_flag.as<int>(),
          c->blk_active.as<int>()); note_launch(); }
      SPH_CUDA(cudaGetLastError());
      SPH_TRY(run_sweep(c, PH_DENSITY, 1, 0, s));
      SPH_CUDA(cudaMemsetAsync(nact, 0, sizeof(int), s));
      { k_hsolve_update<<<div_up(n, TPB), TPB, 0, s>>>(n, hsolve_args(c, nact, nlim)); note_launch(); }
      SPH_CUDA(cudaGetLastError());
      SPH_CUDA(cudaMemcpyAsync(host, nact, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
      SPH_CUDA(cudaStreamSynchronize(s));
      if (total_iters + it < 32) c->stats.newton_active[total_iters + it] = host[0];
      ++it;
      if (host[0] == 0) break;
    }
    if (host[0] == 0) {
      // converged on the host iterations
    } else if (use_dev) {
      int itg = 0;
      SPH_TRY(solve_round_graph(c, s, host, &itg, total_iters + it));
      it += itg;
    } else {
    for (; it < c->prm.max_newton; ++it) {
      SPH_TRY(replan_units(c, 1, nullptr, s));
      { k_block_active<<<div_up((long long)c->nblock * 32, TPB), TPB, 0, s>>>(
          c->nblock, c->b_first.as<int>(), c->b_count.as<int>(), c->h_flag.as<int>(),
          c->blk_active.as<int>()); note_launch(); }
      SPH_CUDA(cudaGetLastError());
      SPH_TRY(run_sweep(c, PH_DENSITY, 1, 0, s));
      SPH_CUDA(cudaMemsetAsync(nact, 0, sizeof(int), s));
      { k_hsolve_update<<<div_up(n, TPB), TPB, 0, s>>>(n, hsolve_args(c, nact, nlim)); note_launch(); }
      SPH_CUDA(cudaGetLastError());
      SPH_CUDA(cudaMemcpyAsync(host, nact, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
      SPH_CUDA(cudaStreamSynchronize(s));
      if (total_iters + it < 32) c->stats.newton_active[total_iters + it] = host[0];
      if (host[0] == 0) {
        ++it;
        break;
      }
    }
    }
    total_iters += it;
    c->stats.unconverged = host[0];
    if (host[0] != 0) {
      c->stats.newton_iters = total_iters;
      return SPH_ERR_H_NOT_CONVERGED;
    }
    if (host[1] == 0) break;
    // positions moved since the build (velocity-Verlet steps) leave the
    // Morton order and build-time positions that an in-place rebuild uses
    // stale: only a full sph_build from the current positions can help
    if (rebuilds >= c->prm.max_rebuild || c->reuse_pad > 0.f) {
      c->stats.newton_iters = total_iters;
      return SPH_ERR_CELL_LIMIT;
    }
    ++rebuilds;
    { k_rebuild_guess<<<div_up(n, TPB), TPB, 0, s>>>(n, c->h.as<float>(), c->hlim.as<float>(),
                                                   c->h_flag.as<int>(), c->nngb.as<float>(),
                                                   c->prm.n_ngb, c->hguess.as<float>()); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    {
      int r = build_from_guess(c, s);
      if (r != SPH_OK) {
        c->built = false;  // the decomposition is half rebuilt
        // no top grid can hold the h this particle set needs (h > box/4)
        return r == SPH_ERR_INVALID_ARG ? SPH_ERR_CELL_LIMIT : r;
      }
    }
    SPH_TRY(ensure_state(c));
    SPH_TRY(prep_mass(c, m, s));
  }
  c->stats.newton_iters = total_iters;
  c->stats.rebuilds = rebuilds;
  if (iters) *iters = total_iters;
  SPH_TRY(compute_node_hmax(c, s));
  const int* perm = c->perm.as<int>();
  // Omega for the caller; the full ghost step runs in sph_force
  { if (h_out) k_scatter<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->h.as<float>(), h_out); note_launch(); }
  { if (rho) k_scatter<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->rho.as<float>(), rho); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  if (omega) {
    { k_ghost<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->h.as<float>(), c->pos4.as<float4>(),
                                           c->rho.as<float>(), c->drho.as<float>(), m, nullptr,
                                           c->prm.gamma, c->omega.as<float>(), c->Avec.as<float>(),
                                           c->u_s.as<float>(), c->vel4.as<float4>(),
                                           c->fdat.as<float4>()); note_launch(); }
    { k_scatter<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->omega.as<float>(), omega); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  c->have_density = true;
  c->have_force = false;
  c->fl_valid = false;
  c->have_d2 = 0;
  return read_status(c, s);
}

int sph_force(sph_ctx* c, const float* u, const float* vel, float* acc, float* dudt,
              int32_t* count, void* stream) {
  if (!c || !u || !acc) return SPH_ERR_INVALID_ARG;
  if (!c->have_density) return SPH_ERR_NOT_BUILT;
  ++c->state_gen;
  cudaStream_t s = as_stream(stream);
  const long long n = c->n;
  const int* perm = c->perm.as<int>();
  { k_ghost<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->h.as<float>(), c->pos4.as<float4>(),
                                         c->rho.as<float>(), c->drho.as<float>(), u, vel,
                                         c->prm.gamma, c->omega.as<float>(), c->Avec.as<float>(),
                                         c->u_s.as<float>(), c->vel4.as<float4>(),
                                         c->fdat.as<float4>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(replan_units(c, 0, nullptr, s));  // the units for the solved h of every particle
  SPH_TRY(run_sweep(c, PH_FORCE, 0, count != nullptr, s));
  { k_scatter_acc<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->acc4.as<float4>(), acc, dudt); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  c->have_force = true;
  if (count) {
    { k_scatter_i<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->cnt_i.as<int>(), count); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    unsigned long long tot = 0;
    SPH_TRY(count_total(c, &tot, s));
    c->stats.force_pairs = (int64_t)(tot / 2);
    return read_status(c, s);
  }
  return SPH_OK;
}

int sph_force_viscous(sph_ctx* c, const float* u, const float* vel, float alpha, float c_cfl,
                      float* acc, float* dudt, float* dt, float* balsara, void* stream) {
  if (!c || !u || !vel || !acc || !dt || !(alpha >= 0.f) || !(c_cfl > 0.f))
    return SPH_ERR_INVALID_ARG;
  if (!c->have_density) return SPH_ERR_NOT_BUILT;
  ++c->state_gen;
  cudaStream_t s = as_stream(stream);
  const long long n = c->n;
  const int* perm = c->perm.as<int>();
  SPH_TRY(dbuf_ensure(c->visc4, 16 * (size_t)n));
  SPH_TRY(dbuf_ensure(c->dt_s, 4 * (size_t)n));
  { k_ghost<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->h.as<float>(), c->pos4.as<float4>(),
                                         c->rho.as<float>(), c->drho.as<float>(), u, vel,
                                         c->prm.gamma, c->omega.as<float>(), c->Avec.as<float>(),
                                         c->u_s.as<float>(), c->vel4.as<float4>(),
                                         c->fdat.as<float4>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  c->visc_alpha = alpha;
  c->visc_cfl = c_cfl;
  SPH_TRY(replan_units(c, 0, nullptr, s));
  SPH_TRY(run_sweep(c, PH_VELDERIV, 0, 0, s));
  SPH_TRY(run_sweep(c, PH_FORCE_VISC, 0, 0, s));
  { k_scatter_acc<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->acc4.as<float4>(), acc, dudt); note_launch(); }
  { k_scatter<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->dt_s.as<float>(), dt); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  if (balsara) {
    { k_scatter_z<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->visc4.as<float4>(), balsara); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  // the adjoints cover the inviscid force only
  c->have_force = false;
  c->fl_valid = false;
  return SPH_OK;
}

int sph_pairs_dump(sph_ctx* c, int32_t phase, int64_t cap, int32_t* pi, int32_t* pj,
                   int64_t* n_out, void* stream) {
  if (!c || !pi || !pj || !n_out || cap < 0 || (phase != 0 && phase != 1))
    return SPH_ERR_INVALID_ARG;
  if (!c->have_density) return SPH_ERR_NOT_BUILT;
  cudaStream_t s = as_stream(stream);
  c->dump_pi = pi;
  c->dump_pj = pj;
  c->dump_cap = cap;
  SPH_CUDA(cudaMemsetAsync(c->counters.p, 0, sizeof(unsigned long long), s));
  if (phase == 1) SPH_TRY(compute_node_hmax(c, s));
  SPH_TRY(run_sweep(c, phase == 0 ? PH_DUMP_DENSITY : PH_DUMP_FORCE, 0, 0, s));
  unsigned long long nn = 0;
  SPH_CUDA(cudaMemcpyAsync(&nn, c->counters.p, sizeof(nn), cudaMemcpyDeviceToHost, s));
  SPH_CUDA(cudaStreamSynchronize(s));
  c->dump_pi = c->dump_pj = nullptr;
  *n_out = (int64_t)nn;
  if ((long long)nn > cap) return SPH_ERR_CAPACITY;
  return read_status(c, s);
}

int sph_set_sweep_config(sph_ctx* c, int32_t warps_per_cta, int32_t sweep_cap,
                         int32_t ctas_per_sm) {
  if (!c || warps_per_cta < 1 || warps_per_cta > 8 || sweep_cap < 32 || sweep_cap > 1024 ||
      (sweep_cap % 32) != 0 || ctas_per_sm < 0)
    return SPH_ERR_INVALID_ARG;
  c->prm.warps_per_cta = warps_per_cta;
  c->prm.sweep_cap = sweep_cap;
  c->sweep_cap = sweep_cap;
  c->prm.ctas_per_sm = ctas_per_sm;
  ++c->build_gen;  // captured graphs hold the old launch shape
  return SPH_OK;
}

int sph_profile(sph_ctx* c, int32_t enable) {
  if (!c) return SPH_ERR_INVALID_ARG;
  SPH_TRY(prof_resolve(c));
  for (int k = 0; k < 8; ++k) {
    c->prof_ms[k] = 0;
    c->prof_n[k] = 0;
    c->prof_units_acc[k] = 0;
    c->prof_cand_acc[k] = 0;
    c->prof_gath_acc[k] = 0;
    c->prof_build_ms[k] = 0;
  }
  c->prof_builds = 0;
  if (enable) SPH_TRY(dbuf_ensure(c->prof_units, 4 * 2048 * sizeof(unsigned long long)));
  c->profile = enable != 0;
  return SPH_OK;
}

int sph_get_stats(sph_ctx* c, sph_stats* out) {
  if (!c || !out) return SPH_ERR_INVALID_ARG;
  SPH_TRY(prof_resolve(c));
  sph_stats st = c->stats;
  for (int k = 0; k < 8; ++k) {
    st.sweep_ms[k] = c->prof_ms[k];
    st.sweep_launches[k] = c->prof_n[k];
    st.sweep_units[k] = (int64_t)c->prof_units_acc[k];
    st.sweep_candidates[k] = (int64_t)c->prof_cand_acc[k];
    st.sweep_gathered[k] = (int64_t)c->prof_gath_acc[k];
  }
  for (int k = 0; k < 8; ++k) st.build_ms[k] = c->prof_build_ms[k];
  st.builds = c->prof_builds;
  st.sweep_grid = c->sweep_grid;
  st.sweep_threads = c->sweep_threads;
  st.n = c->n;
  st.nbox = c->nbox;
  st.ncell = c->ncell;
  if (c->built && c->nleaf_dev.p) {
    int nl = 0;
    SPH_CUDA(cudaDeviceSynchronize());
    SPH_CUDA(cudaMemcpy(&nl, c->nleaf_dev.p, sizeof(int), cudaMemcpyDeviceToHost));
    c->nleaf = nl;
  }
  st.nleaf = c->nleaf;
  st.nblock = c->nblock;
  st.nself = c->nself;
  st.npair = c->npair;
  st.ndt = c->ndt;
  st.max_depth = c->max_depth;
  for (int b = 0; b < 8; ++b) st.top_level[b] = b < c->nbox ? c->box_t[b] : 0;
  st.sorted_entries = c->sorted_entries;
  st.pairs_unlisted = 0;
  st.pairs_unlisted_cut = 0;
  if (c->fl_valid && c->fl_over.p) {
    int ov[2] = {0, 0};
    SPH_CUDA(cudaDeviceSynchronize());
    SPH_CUDA(cudaMemcpy(ov, c->fl_over.p, sizeof(ov), cudaMemcpyDeviceToHost));
    st.pairs_unlisted = ov[0];
    st.pairs_unlisted_cut = ov[1];
  }
  *out = st;
  return SPH_OK;
}

int sph_sync_status(sph_ctx* c, void* stream) {
  if (!c) return SPH_ERR_INVALID_ARG;
  return read_status(c, as_stream(stream));
}

int64_t sph_launch_count(void) { return (int64_t)launch_count(); }

int64_t sph_state_generation(const sph_ctx* c) { return c ? (int64_t)c->state_gen : -1; }

const char* sph_status_string(int st) {
  switch (st) {
    case SPH_OK: return "ok";
    case SPH_ERR_INVALID_ARG: return "invalid argument";
    case SPH_ERR_CUDA: return "CUDA runtime error";
    case SPH_ERR_OOM: return "device out of memory";
    case SPH_ERR_H_NOT_CONVERGED: return "smoothing-length iteration did not converge";
    case SPH_ERR_CELL_LIMIT: return "smoothing length exceeds the cell decomposition";
    case SPH_ERR_NOT_BUILT: return "decomposition or density state missing";
    case SPH_ERR_TIMEOUT: return "bounded device wait timed out";
    case SPH_ERR_CAPACITY: return "output capacity exceeded";
    default: return "unknown status";
  }
}

}  // extern "C"
