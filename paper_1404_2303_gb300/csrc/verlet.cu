// Velocity-Verlet time step (Section 4.1) over the density + force path,
// reusing the decomposition and its sorted lists while the particles have
// moved little since it was built.
//
// A step is kick-drift-kick with one global step: forces at the current
// state, half kick, drift, forces at the new positions with the velocities
// and energies predicted to the end of the step (du/dt and the viscous
// terms depend on them), closing half kick.  Every force evaluation solves
// h afresh, starting from the last solved h.
//
// Reuse (the role of the paper's pseudo-Verlet lists): a decomposition
// built for h (1 + slack) covers every pair r < h_i + 2 d where d is the
// largest displacement since the build, because two particles that moved
// by at most d each were at most 2 d farther apart at the build.  So while
// 2 d stays below the smallest margin hlim_i - h_i, the cells, tasks and
// sorted lists are kept: only the cell-relative positions are refreshed,
// the sweeps widen their axial cutoff and box tests by 2 d (the stored
// sort keys and bounding boxes are stale by at most d), and the h solve
// treats hlim_i - 2 d as the cell limit.  Otherwise, or when a solved h
// outgrows that limit, the decomposition is rebuilt from the current
// positions for h (1 + slack).
#include <cmath>
#include <cstring>

#include "geom.cuh"
#include "internal.cuh"

namespace {

constexpr int TPB = 256;

__device__ __forceinline__ double wrap_box(double x, double L) {
  double w = x - L * floor(x / L);
  if (w >= L) w -= L;
  if (w < 0) w = 0;
  return w;
}

// half kick, drift and prediction: vh = v + dt/2 a, uh = u + dt/2 du,
// x += dt vh (wrapped), vp = vh + dt/2 a, up = uh + dt/2 du
__global__ void k_vv_kick_drift(long long n, double* pos, float* vel, float* u, const float* acc,
                                const float* du, double dt, double L, float* vp, float* up) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float hdt = (float)(0.5 * dt);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float a = acc[3 * p + k];
    const float vh = fmaf(hdt, a, vel[3 * p + k]);
    vel[3 * p + k] = vh;
    vp[3 * p + k] = fmaf(hdt, a, vh);
    pos[3 * p + k] = wrap_box(pos[3 * p + k] + dt * (double)vh, L);
  }
  const float uh = fmaf(hdt, du[p], u[p]);
  u[p] = uh;
  up[p] = fmaf(hdt, du[p], uh);
}

// closing half kick
__global__ void k_vv_kick(long long n, float* vel, float* u, const float* acc, const float* du,
                          double dt) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float hdt = (float)(0.5 * dt);
#pragma unroll
  for (int k = 0; k < 3; ++k) vel[3 * p + k] = fmaf(hdt, acc[3 * p + k], vel[3 * p + k]);
  u[p] = fmaf(hdt, du[p], u[p]);
}

// Positions moved without rebuilding: new top-cell-relative positions (the
// top cell of each particle is the one it was binned into at the build,
// taken by the minimum image), the largest displacement since the build,
// and the smallest margin hlim - h.  Both reductions use the order of
// non-negative floats' bit patterns.
__global__ void k_vv_reuse(long long n, const int* perm, const double* pos, const double* xs,
                           const unsigned long long* keys, double L, int t, int K, const float* h,
                           const float* hlim, float4* pos4, unsigned* d2max, unsigned* marg) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const long long p = perm[s];
  const unsigned long long tm = (keys[s] >> (3 * (K - t))) & ((1ull << (3 * t)) - 1);
  const int ix = compact3(tm >> 2), iy = compact3(tm >> 1), iz = compact3(tm);
  const double e = ldexp(L, -t);
  const int io[3] = {ix, iy, iz};
  float rel[3];
  double d2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double x = pos[3 * p + k];
    double d = x - xs[3 * s + k];
    d -= L * rint(d / L);
    d2 += d * d;
    double r = x - io[k] * e;
    r -= L * rint(r / L - 0.5 * e / L);  // minimum image about the cell centre
    rel[k] = (float)r;
  }
  float4 q = pos4[s];
  q.x = rel[0];
  q.y = rel[1];
  q.z = rel[2];
  pos4[s] = q;
  atomicMax(d2max, __float_as_uint((float)d2));
  const float mg = fmaxf(hlim[s] - h[s], 0.f);
  atomicMin(marg, __float_as_uint(mg));
}

// build guess h (1 + slack), kept below a quarter of the box (the smallest
// top grid has four cells per axis; a root beyond it is reported by the
// solve as a cell limit)
__global__ void k_vv_guess(long long n, const float* h, float f, float hcap, float* out) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p < n) out[p] = fminf(h[p] * f, hcap);
}

__global__ void k_scale_h(long long n, float* h, float f) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s < n) h[s] *= f;
}

__global__ void k_vv_min(long long n, const float* v, unsigned* out) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p < n && v[p] > 0.f) atomicMin(out, __float_as_uint(v[p]));
}

// a decomposition for h (1 + slack) from the current positions; the solve
// then starts from h itself
int vv_build(sph_ctx* c, long long n, const double* pos, double box, float slack, int* nb,
             cudaStream_t s) {
  const float* hg = nullptr;
  if (c->vv_ready) {
    { k_vv_guess<<<div_up(n, TPB), TPB, 0, s>>>(n, c->vv_h.as<float>(), 1.f + slack,
                                                 (float)(0.25 * box) * (1.f - 1e-6f),
                                                 c->vv_tmp.as<float>()); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    hg = c->vv_tmp.as<float>();
  }
  SPH_TRY(sph_build(c, n, pos, box, hg, s));
  if (hg) {
    { k_scale_h<<<div_up(n, TPB), TPB, 0, s>>>(n, c->h.as<float>(), 1.f / (1.f + slack)); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  ++*nb;
  return SPH_OK;
}

// forces (with the viscous terms and the time step of Eq. (dt)) at one
// state, into vv_acc / vv_du / vv_dt (caller order)
int vv_forces(sph_ctx* c, long long n, const double* pos, const float* vel, const float* u,
              const float* m, double box, float alpha, float c_cfl, float slack, int* nb,
              cudaStream_t s) {
  bool reuse = false;
  if (c->built && c->vv_ready && c->n == n && c->nbox == 1 && c->box_L[0] == box) {
    unsigned* red = c->vv_red.as<unsigned>();
    const unsigned init[2] = {0u, 0x7f7fffffu};
    SPH_CUDA(cudaMemcpyAsync(red, init, sizeof(init), cudaMemcpyHostToDevice, s));
    { k_vv_reuse<<<div_up(n, TPB), TPB, 0, s>>>(
        n, c->perm.as<int>(), pos, c->xs.as<double>(), c->keys.as<unsigned long long>(), box,
        c->box_t[0], c->kbits, c->h.as<float>(), c->hlim.as<float>(), c->pos4.as<float4>(), red,
        red + 1); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    unsigned hr[2];
    SPH_CUDA(cudaMemcpyAsync(hr, red, sizeof(hr), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    float d2, mg;
    std::memcpy(&d2, &hr[0], 4);
    std::memcpy(&mg, &hr[1], 4);
    const float pad = 2.f * sqrtf(d2) * (1.f + 1e-5f);
    if (pad < mg) {
      reuse = true;
      if (pad != c->reuse_pad) ++c->build_gen;  // captured graphs hold the margins as arguments
      c->reuse_pad = pad;
    }
  }
  if (!reuse) SPH_TRY(vv_build(c, n, pos, box, slack, nb, s));
  int r;
  {
    const int saved = c->prm.max_rebuild;
    if (reuse) c->prm.max_rebuild = 0;  // the in-place rebuild assumes build-time positions
    r = sph_density(c, m, c->vv_h.as<float>(), nullptr, nullptr, nullptr, s);
    c->prm.max_rebuild = saved;
  }
  if (reuse && r == SPH_ERR_CELL_LIMIT) {
    // a solved h outgrew the reduced cell limit: rebuild from the current
    // positions, cells sized from the density estimate
    c->vv_ready = false;
    SPH_TRY(sph_build(c, n, pos, box, nullptr, s));
    ++*nb;
    r = sph_density(c, m, c->vv_h.as<float>(), nullptr, nullptr, nullptr, s);
  }
  if (r != SPH_OK) return r;
  c->vv_ready = true;
  return sph_force_viscous(c, u, vel, alpha, c_cfl, c->vv_acc.as<float>(), c->vv_du.as<float>(),
                           c->vv_dt.as<float>(), nullptr, s);
}

}  // namespace

extern "C" int sph_verlet_step(sph_ctx* c, int64_t n, double* pos, float* vel, float* u,
                               const float* m, double box, double dt, float alpha, float c_cfl,
                               float slack, float* dt_min, int32_t* rebuilt, void* stream) {
  if (!c || n <= 0 || !pos || !vel || !u || !m || !(box > 0) || !(dt > 0) || !(alpha >= 0.f) ||
      !(c_cfl > 0.f) || !(slack > 0.f) || slack > 1.f)
    return SPH_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (c->n != n || !c->built) c->vv_ready = false;
  const size_t N = (size_t)n;
  SPH_TRY(dbuf_ensure(c->vv_acc, 12 * N));
  SPH_TRY(dbuf_ensure(c->vv_vp, 12 * N));
  SPH_TRY(dbuf_ensure(c->vv_du, 4 * N));
  SPH_TRY(dbuf_ensure(c->vv_dt, 4 * N));
  SPH_TRY(dbuf_ensure(c->vv_up, 4 * N));
  SPH_TRY(dbuf_ensure(c->vv_h, 4 * N));
  SPH_TRY(dbuf_ensure(c->vv_tmp, 4 * N));
  SPH_TRY(dbuf_ensure(c->vv_red, 64));
  int nb = 0;
  SPH_TRY(vv_forces(c, n, pos, vel, u, m, box, alpha, c_cfl, slack, &nb, s));
  { k_vv_kick_drift<<<div_up(n, TPB), TPB, 0, s>>>(n, pos, vel, u, c->vv_acc.as<float>(),
                                                    c->vv_du.as<float>(), dt, box,
                                                    c->vv_vp.as<float>(), c->vv_up.as<float>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(vv_forces(c, n, pos, c->vv_vp.as<float>(), c->vv_up.as<float>(), m, box, alpha, c_cfl,
                    slack, &nb, s));
  { k_vv_kick<<<div_up(n, TPB), TPB, 0, s>>>(n, vel, u, c->vv_acc.as<float>(), c->vv_du.as<float>(),
                                              dt); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  if (dt_min) {
    unsigned* red = c->vv_red.as<unsigned>() + 2;
    const unsigned init = 0x7f7fffffu;
    SPH_CUDA(cudaMemcpyAsync(red, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    { k_vv_min<<<div_up(n, TPB), TPB, 0, s>>>(n, c->vv_dt.as<float>(), red); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    unsigned hv = 0;
    SPH_CUDA(cudaMemcpyAsync(&hv, red, sizeof(hv), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    std::memcpy(dt_min, &hv, 4);
  }
  if (rebuilt) *rebuilt = nb;
  return SPH_OK;
}
