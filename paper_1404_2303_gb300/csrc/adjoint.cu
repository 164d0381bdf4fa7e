// Reverse mode of the SPH step (the paper has no adjoint; this is the
// chain rule through Eq. (dvdt), (dudt), the ghost quantities of Section
// 2.1, Eq. (rho) and the implicit smoothing length of Eq. (nneigh)).
// The adjoint sweeps recompute every pair term from positions instead of
// storing neighbour lists.
#include "internal.cuh"

namespace {

constexpr int TPB = 256;
constexpr float SIGMA = 2.546479089470325f;  // 8/pi

__global__ void k_gather_gacc(long long n, const int* perm, const float* g_acc,
                              const float* g_dudt, float4* adj4) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  long long p = perm[s];
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (g_acc) {
    v.x = g_acc[3 * p];
    v.y = g_acc[3 * p + 1];
    v.z = g_acc[3 * p + 2];
  }
  if (g_dudt) v.w = g_dudt[p];
  adj4[s] = v;
}

// ghost step reversed: A = (gamma-1) u / (Omega rho), Omega = 1 + h rho'/(3 rho)
__global__ void k_ghost_adj(long long n, const float* h, const float* rho, const float* drho,
                            const float* omega, const float* A, float gamma, const float* gA,
                            const float* ghraw, float* g_u, float* g_rho, float* g_drho,
                            float* g_h) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  float r = rho[s], om = omega[s], a = A[s], hv = h[s], rp = drho[s], ga = gA[s];
  float gO = -ga * a / om;
  g_u[s] = ga * (gamma - 1.f) / (om * r);
  g_rho[s] = -ga * a / r - gO * hv * rp / (3.f * r * r);
  g_drho[s] = gO * hv / (3.f * r);
  g_h[s] = a * ghraw[s] + gO * rp / (3.f * r);
}

// per-particle data of the density adjoint sweep (see PDensityAdj)
__global__ void k_dens_adj_prep(long long n, const float* h, const float* drho, const float* d2rho,
                                const float* dnngb, const float* g_rho, const float* g_drho,
                                const float* g_h, float4* adj4, float4* adj4b) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float hv = h[s];
  float hi = 1.f / hv;
  float hi2 = hi * hi, hi3 = hi2 * hi, hi4 = hi2 * hi2;
  float gr = g_rho[s], grp = g_drho[s];
  float ghtot = g_h[s] + gr * drho[s] + grp * d2rho[s];
  float lam = ghtot / dnngb[s];
  adj4[s] = make_float4(hi, 2.f * SIGMA * hi3 * gr, 6.f * SIGMA * hi4 * grp, 6.f * SIGMA * hi4 * gr);
  adj4b[s] = make_float4(SIGMA * hi4 * hi * grp, 64.f * lam * hi, __fmul_rn(hv, hv), 0.f);
}

__global__ void k_gather_f(long long n, const int* perm, const float* in, float* out, int add) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  float v = in ? in[perm[s]] : 0.f;
  out[s] = add ? out[s] + v : v;
}

__global__ void k_scatter_f(long long n, const int* perm, const float* in, float* out) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s < n) out[perm[s]] = in[s];
}

__global__ void k_scatter_gx(long long n, const int* perm, const float4* gx4, float* g_pos,
                             float* g_m, int add) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  long long p = perm[s];
  float4 g = gx4[s];
  if (add) {
    g_pos[3 * p] += g.x;
    g_pos[3 * p + 1] += g.y;
    g_pos[3 * p + 2] += g.z;
    if (g_m) g_m[p] += g.w;
  } else {
    g_pos[3 * p] = g.x;
    g_pos[3 * p + 1] = g.y;
    g_pos[3 * p + 2] = g.z;
    if (g_m) g_m[p] = g.w;
  }
}

int ensure_adj(sph_ctx* c) {
  const size_t n = (size_t)c->n;
  SPH_TRY(dbuf_ensure(c->adj4, 16 * n));
  SPH_TRY(dbuf_ensure(c->adj4b, 16 * n));
  SPH_TRY(dbuf_ensure(c->g_x4, 16 * n));
  DBuf* f[] = {&c->g_A, &c->g_rho_s, &c->g_drho_s, &c->g_h_s, &c->g_u_s};
  for (DBuf* b : f) SPH_TRY(dbuf_ensure(*b, 4 * n));
  return SPH_OK;
}

int force_adj_internal(sph_ctx* c, const float* g_acc, const float* g_dudt, cudaStream_t s) {
  const long long n = c->n;
  { k_gather_gacc<<<div_up(n, TPB), TPB, 0, s>>>(n, c->perm.as<int>(), g_acc, g_dudt,
                                               c->adj4.as<float4>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(run_sweep(c, PH_FORCE_ADJ, 0, 0, s));
  { k_ghost_adj<<<div_up(n, TPB), TPB, 0, s>>>(
      n, c->h.as<float>(), c->rho.as<float>(), c->drho.as<float>(), c->omega.as<float>(),
      c->Avec.as<float>(), c->prm.gamma, c->g_A.as<float>(), c->g_h_s.as<float>(),
      c->g_u_s.as<float>(), c->g_rho_s.as<float>(), c->g_drho_s.as<float>(), c->g_h_s.as<float>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  return SPH_OK;
}

int density_adj_internal(sph_ctx* c, cudaStream_t s) {
  const long long n = c->n;
  if (!c->have_d2) {
    SPH_TRY(run_sweep(c, PH_DENSITY_D2, 0, 0, s));
    c->have_d2 = 1;
  }
  { k_dens_adj_prep<<<div_up(n, TPB), TPB, 0, s>>>(
      n, c->h.as<float>(), c->drho.as<float>(), c->d2rho.as<float>(), c->dnngb.as<float>(),
      c->g_rho_s.as<float>(), c->g_drho_s.as<float>(), c->g_h_s.as<float>(), c->adj4.as<float4>(),
      c->adj4b.as<float4>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(run_sweep(c, PH_DENSITY_ADJ, 0, 0, s));
  return SPH_OK;
}

}  // namespace

static cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" {

int sph_force_adjoint(sph_ctx* c, const float* g_acc, const float* g_dudt, float* g_pos,
                      float* g_m, float* g_u, float* g_rho, float* g_drho, float* g_h,
                      void* stream) {
  if (!c || !g_acc || !g_pos || !g_m || !g_u || !g_rho || !g_drho || !g_h)
    return SPH_ERR_INVALID_ARG;
  if (!c->have_force) return SPH_ERR_NOT_BUILT;
  cudaStream_t s = as_stream(stream);
  const long long n = c->n;
  const int* perm = c->perm.as<int>();
  SPH_TRY(ensure_adj(c));
  SPH_TRY(force_adj_internal(c, g_acc, g_dudt, s));
  { k_scatter_gx<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->g_x4.as<float4>(), g_pos, g_m, 0); note_launch(); }
  { k_scatter_f<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->g_u_s.as<float>(), g_u); note_launch(); }
  { k_scatter_f<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->g_rho_s.as<float>(), g_rho); note_launch(); }
  { k_scatter_f<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->g_drho_s.as<float>(), g_drho); note_launch(); }
  { k_scatter_f<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->g_h_s.as<float>(), g_h); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  return SPH_OK;
}

int sph_density_adjoint(sph_ctx* c, const float* g_rho, const float* g_drho, const float* g_h,
                        float* g_pos, float* g_m, void* stream) {
  if (!c || !g_rho || !g_pos || !g_m) return SPH_ERR_INVALID_ARG;
  if (!c->have_density) return SPH_ERR_NOT_BUILT;
  cudaStream_t s = as_stream(stream);
  const long long n = c->n;
  const int* perm = c->perm.as<int>();
  SPH_TRY(ensure_adj(c));
  { k_gather_f<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, g_rho, c->g_rho_s.as<float>(), 0); note_launch(); }
  { k_gather_f<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, g_drho, c->g_drho_s.as<float>(), 0); note_launch(); }
  { k_gather_f<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, g_h, c->g_h_s.as<float>(), 0); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_CUDA(cudaMemsetAsync(c->g_x4.p, 0, 16 * (size_t)n, s));
  SPH_TRY(density_adj_internal(c, s));
  { k_scatter_gx<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->g_x4.as<float4>(), g_pos, g_m, 1); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  return SPH_OK;
}

int sph_adjoint(sph_ctx* c, const float* g_rho, const float* g_acc, const float* g_dudt,
                float* g_pos, float* g_m, float* g_u, void* stream) {
  if (!c || !g_pos || !g_m || !g_u) return SPH_ERR_INVALID_ARG;
  if (!c->have_density) return SPH_ERR_NOT_BUILT;
  cudaStream_t s = as_stream(stream);
  const long long n = c->n;
  const int* perm = c->perm.as<int>();
  SPH_TRY(ensure_adj(c));
  if (g_acc || g_dudt) {
    if (!c->have_force) return SPH_ERR_NOT_BUILT;
    SPH_TRY(force_adj_internal(c, g_acc, g_dudt, s));
  } else {
    SPH_CUDA(cudaMemsetAsync(c->g_x4.p, 0, 16 * (size_t)n, s));
    DBuf* z[] = {&c->g_rho_s, &c->g_drho_s, &c->g_h_s, &c->g_u_s};
    for (DBuf* b : z) SPH_CUDA(cudaMemsetAsync(b->p, 0, 4 * (size_t)n, s));
  }
  if (g_rho) {
    { k_gather_f<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, g_rho, c->g_rho_s.as<float>(), 1); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  SPH_TRY(density_adj_internal(c, s));
  { k_scatter_gx<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->g_x4.as<float4>(), g_pos, g_m, 0); note_launch(); }
  { k_scatter_f<<<div_up(n, TPB), TPB, 0, s>>>(n, perm, c->g_u_s.as<float>(), g_u); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  return SPH_OK;
}

}  // extern "C"
