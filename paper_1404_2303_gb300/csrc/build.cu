// Decomposition build: Morton order, the hierarchical cells of Section 3.2,
// the self/pair task refinement of Fig. SplitCell / SplitPair, per-warp
// particle blocks, the 13-direction sorted lists of Section 3.3 (blocks
// sorted in shared memory, parents merged from their sub-cells as in
// Fig. HierarchySorting) and the per-block interaction lists the sweeps
// consume.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include <chrono>

#include "geom.cuh"
#include "internal.cuh"

namespace {

constexpr int TPB = 256;
constexpr int EST_SPLIT = 64;  // count-only split threshold of the h-estimate octree

__device__ __forceinline__ int box_of(const long long* off, int nbox, long long p) {
  int lo = 0, hi = nbox;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int box_of_node(const int* top_base, int nbox, int id) {
  int lo = 0, hi = nbox;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (top_base[mid] <= id) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double wrap_pos(double x, double L) {
  if (x >= 0.0 && x < L) return x;  // inside the box already (no FP64 division)
  double w = x - L * floor(x / L);
  if (w >= L) w -= L;
  if (w < 0) w = 0;
  return w;
}

__device__ __forceinline__ int lower_bound_u64(const unsigned long long* a, int lo, int hi,
                                               unsigned long long v) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------- keys
__global__ void k_keys(const double* pos, long long n, const long long* off, const double* Ls,
                       int nbox, int K, unsigned long long* keys, int* perm, int* status) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= n) return;
  int b = box_of(off, nbox, p);
  double L = Ls[b];
  double scale = (double)(1u << K) / L;
  unsigned q[3];
  for (int k = 0; k < 3; ++k) {
    const double x0 = pos[3 * p + k];
    if (!isfinite(x0)) atomicOr(status, ST_BAD_INPUT);  // reported by the build; key clamped below
    double x = isfinite(x0) ? wrap_pos(x0, L) : 0.0;
    long long v = (long long)floor(x * scale);
    v = v < 0 ? 0 : (v > (1ll << K) - 1 ? (1ll << K) - 1 : v);
    q[k] = (unsigned)v;
  }
  keys[p] = ((unsigned long long)b << (3 * K)) | morton3(q[0], q[1], q[2]);
  perm[p] = (int)p;
}

__global__ void k_gather_pos(const double* pos, const int* perm, long long n, const long long* off,
                             const double* Ls, int nbox, const float* hg_in, double* xs,
                             float* hg_out, int* status) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  int p = perm[s];
  int b = box_of(off, nbox, p);
  double L = Ls[b];
  for (int k = 0; k < 3; ++k) {
    const double x0 = pos[3 * (long long)p + k];
    xs[3 * s + k] = isfinite(x0) ? wrap_pos(x0, L) : 0.0;
  }
  if (hg_in) {
    float g = hg_in[p];
    if (!(g > 0.f) || !isfinite(g)) {  // a guess must be a positive finite length
      atomicOr(status, ST_BAD_INPUT);
      g = (float)(0.25 * L);
    }
    hg_out[s] = g;
  }
}

// ---------------------------------------------------------------- octree
struct NodeArrays {
  int *first, *count, *parent, *child0, *top, *box;
  int4* ijk;
  float* hbuild;
};

__global__ void k_init_top(int ntop, const int* top_base, const int* box_t, int nbox,
                           const unsigned long long* keys, int n, int K, NodeArrays na) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= ntop) return;
  int b = box_of_node(top_base, nbox, id);
  int t = box_t[b];
  int nb = 1 << t;
  int loc = id - top_base[b];
  int ix = loc / (nb * nb), iy = (loc / nb) % nb, iz = loc % nb;
  unsigned long long m = morton3(ix, iy, iz);
  int sh = 3 * (K - t);
  unsigned long long lo = ((unsigned long long)b << (3 * K)) | (m << sh);
  unsigned long long hi = lo + (1ull << sh);
  int f = lower_bound_u64(keys, 0, n, lo);
  int e = lower_bound_u64(keys, f, n, hi);
  na.first[id] = f;
  na.count[id] = e - f;
  na.parent[id] = -1;
  na.child0[id] = -1;
  na.top[id] = id;
  na.box[id] = b;
  na.ijk[id] = make_int4(ix, iy, iz, t);
}


// structural fields of the 8 children of each split node; their particle
// ranges are filled by k_pcur_update from the Morton-key boundaries
// children of the splitting nodes of the generation, placed after it in
// split order; ctl[2] is set (and nothing created) when they would not fit
__global__ void k_make_children(int* ctl, int ngmax, int cap, const int* split, const int* soff,
                                NodeArrays na, int* acc_h, int* acc_s, int* cend) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int g0 = ctl[0], g1 = ctl[1];
  if ((long long)g1 + 8ll * soff[ngmax] > (long long)cap) {
    if (i == 0) ctl[2] = 1;
    return;
  }
  const int node = g0 + i;
  if (i >= ngmax || node >= g1 || !split[i]) return;
  int c0 = g1 + 8 * soff[i];
  na.child0[node] = c0;
  int4 p = na.ijk[node];
  int b = na.box[node];
  int lvl = p.w + 1;
  for (int k = 0; k < 8; ++k) {
    int cx = 2 * p.x + ((k >> 2) & 1), cy = 2 * p.y + ((k >> 1) & 1), cz = 2 * p.z + (k & 1);
    int id = c0 + k;
    na.first[id] = 0;
    na.count[id] = 0;
    na.parent[id] = node;
    na.child0[id] = -1;
    na.top[id] = na.top[node];
    na.box[id] = b;
    na.ijk[id] = make_int4(cx, cy, cz, lvl);
    acc_h[id] = 0;
    acc_s[id] = 0;
    cend[id] = 0;
  }
}

// h estimate from a count-only octree below a 4^3 top grid whose cells
// split above EST_SPLIT particles: the local number density of the
// particle's leaf's parent (or of the leaf itself at the top level; in mode 1
// the lower of the leaf's and the parent's), turned into the h whose sphere
// holds N_ngb particles at that density.  The octree is not built: in the
// sorted Morton keys the particles of the level-L cell holding particle s
// form one run of equal key prefixes, so the leaf (the first level whose cell
// holds at most EST_SPLIT particles) and its parent are found by binary
// searches over the level and over the run ends.
__device__ __forceinline__ long long first_ge(const unsigned long long* keys, long long a, long long b,
                                              unsigned long long P, int sh) {
  while (a < b) {  // first index in [a, b) whose prefix is >= P
    const long long m = (a + b) >> 1;
    if ((keys[m] >> sh) < P) a = m + 1; else b = m;
  }
  return a;
}
__device__ __forceinline__ long long first_gt(const unsigned long long* keys, long long a, long long b,
                                              unsigned long long P, int sh) {
  while (a < b) {  // first index in [a, b) whose prefix is > P
    const long long m = (a + b) >> 1;
    if ((keys[m] >> sh) <= P) a = m + 1; else b = m;
  }
  return a;
}

__global__ void k_h_estimate_flat(long long n, const unsigned long long* keys, int K, int t0,
                                  const double* Ls, float n_ngb, int mode, float factor,
                                  float* hout) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const unsigned long long key = keys[s];
  const int b = (int)(key >> (3 * K));
  // run length of s's level-L cell, exact when at most EST_SPLIT (else > EST_SPLIT)
  auto small_count = [&](int L) -> long long {
    const int sh = 3 * (K - L);
    const unsigned long long P = key >> sh;
    const long long a = s - EST_SPLIT > 0 ? s - EST_SPLIT : 0;
    const long long e = s + EST_SPLIT + 1 < n ? s + EST_SPLIT + 1 : n;
    return first_gt(keys, s + 1, e, P, sh) - first_ge(keys, a, s, P, sh);
  };
  int lo = t0, hi = K;  // first level whose cell holds <= EST_SPLIT (K at most)
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (small_count(mid) <= EST_SPLIT) hi = mid; else lo = mid + 1;
  }
  const int Ll = lo;
  const double L = Ls[b];
  const int shl = 3 * (K - Ll);
  const long long cl = first_gt(keys, s + 1, n, key >> shl, shl) - first_ge(keys, 0, s, key >> shl, shl);
  // number densities count / edge^3 with edge = L 2^-level (FP32 suffices
  // for an estimate)
  const float iv = 1.0f / (float)(L * L * L);
  float dens = (float)cl * ldexpf(iv, 3 * Ll);
  if (Ll > t0) {
    const int Lp = Ll - 1, shp = 3 * (K - Lp);
    const long long cp = first_gt(keys, s + 1, n, key >> shp, shp) - first_ge(keys, 0, s, key >> shp, shp);
    const float dp = (float)cp * ldexpf(iv, 3 * Lp);
    dens = (mode == 1 && cl >= 8) ? fminf(dp, dens) : dp;
  }
  const float h = factor * cbrtf((float)(3.0 * (double)n_ngb / (4.0 * M_PI)) / dens);
  hout[s] = fminf(h, (float)(0.24 * L));
}

__global__ void k_scale(long long n, float* v, float f) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s < n) v[s] *= f;
}

__global__ void k_relpos(long long n, const unsigned long long* keys, const double* xs,
                         const double* Ls, const int* box_t, int K, float4* pos4, float* p_et) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  unsigned long long key = keys[s];
  int b = (int)(key >> (3 * K));
  int t = box_t[b];
  unsigned long long tm = (key >> (3 * (K - t))) & ((1ull << (3 * t)) - 1);
  int ix = compact3(tm >> 2), iy = compact3(tm >> 1), iz = compact3(tm);
  double e = ldexp(Ls[b], -t);
  float4 v;
  v.x = (float)(xs[3 * s + 0] - ix * e);
  v.y = (float)(xs[3 * s + 1] - iy * e);
  v.z = (float)(xs[3 * s + 2] - iz * e);
  v.w = 0.f;
  pos4[s] = v;
  p_et[s] = (float)e;
}

// ---------------------------------------------------------------- tasks
// task: int4 {ci, cj, packed offset/periodic image, type (0 self, 1 pair)}
__device__ __forceinline__ int top_id(const int* top_base, int b, int n, int x, int y, int z) {
  return top_base[b] + (x * n + y) * n + z;
}

__global__ void k_top_tasks(int ntop, const int* top_base, const int* box_t, int nbox,
                            const int* count, const int* off, int* cnt, int4* out) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= ntop) return;
  int emitted = 0;
  int base = off ? off[id] : 0;
  if (count[id] > 0) {
    int b = box_of_node(top_base, nbox, id);
    int n = 1 << box_t[b];
    int loc = id - top_base[b];
    int ix = loc / (n * n), iy = (loc / n) % n, iz = loc % n;
    if (out) out[base] = make_int4(id, id, 0, 0);
    emitted = 1;
    for (int d = 0; d < SPH_NDIR; ++d) {
      int ox, oy, oz;
      dir_offset(d, ox, oy, oz);
      int x = ix + ox, y = iy + oy, z = iz + oz;
      int px = x < 0 ? -1 : (x >= n ? 1 : 0);
      int py = y < 0 ? -1 : (y >= n ? 1 : 0);
      int pz = z < 0 ? -1 : (z >= n ? 1 : 0);
      x -= px * n; y -= py * n; z -= pz * n;
      int nb = top_id(top_base, b, n, x, y, z);
      if (count[nb] == 0) continue;
      if (out) out[base + emitted] = make_int4(id, nb, pack_pair(ox, oy, oz, px, py, pz), 1);
      ++emitted;
    }
  }
  if (cnt) cnt[id] = emitted;
}

__device__ __forceinline__ bool pair_splits(int a, int b, const int* child0, const float* hb,
                                            const int4* ijk, const int* box, const double* Ls) {
  if (child0[a] < 0 || child0[b] < 0) return false;
  double e = ldexp(Ls[box[a]], -ijk[a].w);
  float half = (float)(0.5 * e);
  return hb[a] <= half && hb[b] <= half;
}

// count (out == nullptr) or emit the children of each task; final tasks go
// to the self / pair lists.  The task count *ntp and the list lengths so far
// (fin_len: self, pair) live on the device.  In emit mode the offsets come
// from one exclusive scan over [child counts | self counts | pair counts]
// (each cap + 1 long, zero gaps), so the self and pair offsets carry the
// totals before them (off_s[cap], off_p[cap] hold the running sums).
__global__ void k_refine(const int* ntp, int cap, const int4* tasks, const int* child0,
                         const int* count, const float* hb, const int4* ijk, const int* box,
                         const double* Ls, int* nchild, int* nfs, int* nfp, const int* off_c,
                         const int* off_s, const int* off_p, int4* out, int* fin_self,
                         int4* fin_pair, const int* fin_len, int* psplit) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *ntp || t >= cap) return;
  const int fs_base = out ? fin_len[0] - off_c[cap] : 0;
  const int fp_base = out ? fin_len[1] - off_s[cap] : 0;
  int4 tk = tasks[t];
  int nc = 0, fs = 0, fp = 0;
  int oc = off_c ? off_c[t] : 0;
  if (tk.w == 0) {
    int c = tk.x;
    int c0 = child0[c];
    if (c0 < 0) {
      fs = 1;
      if (fin_self) fin_self[fs_base + off_s[t]] = c;
    } else {
      for (int a = 0; a < 8; ++a) {
        int ca = c0 + a;
        if (count[ca] == 0) continue;
        if (out) out[oc + nc] = make_int4(ca, ca, 0, 0);
        ++nc;
        for (int b2 = a + 1; b2 < 8; ++b2) {
          int cb = c0 + b2;
          if (count[cb] == 0) continue;
          int4 ia = ijk[ca], ib = ijk[cb];
          if (out)
            out[oc + nc] = make_int4(ca, cb, pack_pair(ib.x - ia.x, ib.y - ia.y, ib.z - ia.z, 0, 0, 0), 1);
          ++nc;
        }
      }
    }
  } else {
    int a = tk.x, b = tk.y;
    if (!pair_splits(a, b, child0, hb, ijk, box, Ls)) {
      fp = 1;
      if (fin_pair) fin_pair[fp_base + off_p[t]] = tk;
    } else {
      if (psplit) {
        psplit[a] = 1;
        psplit[b] = 1;
      }
      int ox, oy, oz, px, py, pz;
      unpack_pair(tk.z, ox, oy, oz, px, py, pz);
      int a0 = child0[a], b0 = child0[b];
      int n2 = 1 << (ijk[a].w + 1);
      for (int i = 0; i < 8; ++i) {
        int ca = a0 + i;
        if (count[ca] == 0) continue;
        int4 ia = ijk[ca];
        for (int j = 0; j < 8; ++j) {
          int cb = b0 + j;
          if (count[cb] == 0) continue;
          int4 ib = ijk[cb];
          int dx = ib.x + px * n2 - ia.x, dy = ib.y + py * n2 - ia.y, dz = ib.z + pz * n2 - ia.z;
          if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) continue;
          if (out) out[oc + nc] = make_int4(ca, cb, pack_pair(dx, dy, dz, px, py, pz), 1);
          ++nc;
        }
      }
    }
  }
  if (nchild) {
    nchild[t] = nc;
    nfs[t] = fs;
    nfp[t] = fp;
  }
}

// after an emit pass: the next generation's task count and the list lengths
__global__ void k_refine_advance(int cap, const int* off_c, const int* off_s, const int* off_p,
                                 int* ntp, int* fin_len) {
  const int tch = off_c[cap], tcs = off_s[cap], tcp = off_p[cap];
  *ntp = tch;
  fin_len[0] += tcs - tch;
  fin_len[1] += tcp - tcs;
}

__global__ void k_hlim(int g0, int g1, const int* parent, const int* psplit, const int4* ijk,
                       const int* box, const double* Ls, float* hlim) {
  int node = g0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g1) return;
  int p = parent[node];
  double L = Ls[box[node]];
  if (p < 0) {
    hlim[node] = (float)(ldexp(L, -ijk[node].w));
  } else {
    float v = hlim[p];
    if (psplit[p]) v = fminf(v, (float)(0.5 * ldexp(L, -ijk[p].w)));
    hlim[node] = v;
  }
}

__global__ void k_particle_hlim(long long n, const int* pnode, const float* nh, float* ph) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s < n) ph[s] = nh[pnode[s]];
}

// ---------------------------------------------------------------- blocks
__global__ void k_leaf_nblk(int ncell, const int* child0, const int* count, int bmax, int* nblk) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= ncell) return;
  int c = count[id];
  nblk[id] = (child0[id] < 0 && c > 0) ? (c + bmax - 1) / bmax : 0;
}

__global__ void k_make_blocks(int ncell, const int* first, const int* count, const int* nblk,
                              const int* boff, int* b_first, int* b_count, int* b_leaf,
                              int* n_blk0) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= ncell) return;
  int nb = nblk[id];
  n_blk0[id] = nb > 0 ? boff[id] : -1;
  if (nb == 0) return;
  int c = count[id], f = first[id];
  int q = c / nb, r = c % nb;
  for (int k = 0; k < nb; ++k) {
    int bi = boff[id] + k;
    b_first[bi] = f + k * q + min(k, r);
    b_count[bi] = q + (k < r ? 1 : 0);
    b_leaf[bi] = id;
  }
}

// ---------------------------------------------------------------- sorts
// (key, global index) order: ties cannot occur because indices are distinct

__device__ __forceinline__ bool kv_less(float ka, int ia, float kb, int ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// One warp per block sorts it along all 13 directions: the block's
// positions are loaded once (R per lane, padded to 32 R with +inf keys) and
// each direction's (key, index) pairs are sorted by a bitonic network in
// registers: partners 32 or more apart sit in the same lane, closer ones are
// exchanged with shuffles.
constexpr int WS_WARPS = 8;

template <int R>
__device__ __forceinline__ void sort_block_dirs(int f, int c, const float4* pos4, float* s_key,
                                                int* s_idx) {
  const int lane = threadIdx.x & 31;
  constexpr int NP = 32 * R;
  float px[R], py[R], pz[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int t = r * 32 + lane;
    if (t < c) {
      const float4 p = pos4[f + t];
      px[r] = p.x; py[r] = p.y; pz[r] = p.z;
    } else {
      px[r] = py[r] = pz[r] = 0.f;
    }
  }
  for (int d = 0; d < SPH_NDIR; ++d) {
    float ux, uy, uz;
    dir_unit(d, ux, uy, uz);
    float k[R];
    int x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int t = r * 32 + lane;
      k[r] = t < c ? sort_key(px[r], py[r], pz[r], ux, uy, uz) : __int_as_float(0x7f800000);
      x[r] = t < c ? f + t : 0x7fffffff;
    }
#pragma unroll
    for (int kk = 2; kk <= NP; kk <<= 1) {
#pragma unroll
      for (int j = kk >> 1; j > 0; j >>= 1) {
        if (j >= 32) {
          const int js = j >> 5;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            if (r & js) continue;
            const int r2 = r | js;
            const bool up = ((r * 32 + lane) & kk) == 0;
            const bool sw = up ? kv_less(k[r2], x[r2], k[r], x[r]) : kv_less(k[r], x[r], k[r2], x[r2]);
            if (sw) {
              const float tk = k[r]; k[r] = k[r2]; k[r2] = tk;
              const int tx = x[r]; x[r] = x[r2]; x[r2] = tx;
            }
          }
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float ok = __shfl_xor_sync(0xffffffffu, k[r], j);
            const int ox = __shfl_xor_sync(0xffffffffu, x[r], j);
            const bool lower = (lane & j) == 0;
            const bool up = ((r * 32 + lane) & kk) == 0;
            // the lower partner keeps the smaller pair in ascending runs
            const bool other_less = kv_less(ok, ox, k[r], x[r]);
            const bool take = (lower == up) ? other_less : !other_less;
            if (take) { k[r] = ok; x[r] = ox; }
          }
        }
      }
    }
    const long long o = 13ll * f + (long long)d * c;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int t = r * 32 + lane;
      if (t < c) {
        s_key[o + t] = k[r];
        s_idx[o + t] = x[r];
      }
    }
  }
}

__global__ void __launch_bounds__(WS_WARPS * 32)
    k_sort_blocks_warp(int nblock, const int* b_first, const int* b_count, const float4* pos4,
                       float* s_key, int* s_idx) {
  const int warp = threadIdx.x >> 5;
  for (long long b = (long long)blockIdx.x * WS_WARPS + warp; b < nblock;
       b += (long long)gridDim.x * WS_WARPS) {
    const int f = b_first[b], c = b_count[b];
    if (c <= 32) sort_block_dirs<1>(f, c, pos4, s_key, s_idx);
    else if (c <= 64) sort_block_dirs<2>(f, c, pos4, s_key, s_idx);
    else if (c <= 128) sort_block_dirs<4>(f, c, pos4, s_key, s_idx);
    else sort_block_dirs<8>(f, c, pos4, s_key, s_idx);
  }
}

__global__ void k_need_pairs(int np, const int4* pairs, int* need) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= np) return;
  int4 tk = pairs[t];
  int ox, oy, oz, px, py, pz;
  unpack_pair(tk.z, ox, oy, oz, px, py, pz);
  int oc = off_code(ox, oy, oz);
  int d = oc > 13 ? oc - 14 : 12 - oc;
  atomicOr(&need[tk.x], 1 << d);
  atomicOr(&need[tk.y], 1 << d);
}

__global__ void k_need_self(int ncell, const int* nblk, int* need) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id < ncell && nblk[id] > 1) atomicOr(&need[id], 1 << SPH_SELF_DIR);
}

__global__ void k_need_down(int g0, int g1, const int* child0, int* need) {
  int node = g0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g1) return;
  int c0 = child0[node], nd = need[node];
  if (c0 < 0 || nd == 0) return;
  for (int k = 0; k < 8; ++k) atomicOr(&need[c0 + k], nd);
}

// A node is listed (its 13 sorted lists exist) when it holds at most
// list_cap (<= LIST_CAP) particles and every descendant is listed; a leaf
// also needs at most LIST_SUB blocks.  Its lists are then merged in shared memory from its
// children's (or its blocks') lists.  A task that names an unlisted node
// reaches its particles through the listed descendants, or through the
// blocks of an unlisted leaf (blocks always have lists).  ex[node] counts the
// interaction-list entries a reference to the node expands to.
constexpr int LIST_CAP = 4096;
constexpr int LIST_SUB = 16;

__global__ void k_listed(int g0, int g1, const int* child0, const int* count, const int* nblk,
                         int cap, int* listed, int* ex) {
  int node = g0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g1) return;
  const int cnt = count[node];
  if (cnt == 0) {
    listed[node] = 1;
    ex[node] = 0;
    return;
  }
  const int c0 = child0[node];
  if (c0 < 0) {
    const bool L = cnt <= cap && nblk[node] <= LIST_SUB;
    listed[node] = L ? 1 : 0;
    ex[node] = L ? 1 : nblk[node];
    return;
  }
  bool all = cnt <= cap;
  int e = 0;
  for (int k = 0; k < 8; ++k) {
    all = all && listed[c0 + k] != 0;
    e += ex[c0 + k];
  }
  listed[node] = all ? 1 : 0;
  ex[node] = all ? 1 : e;
}

__global__ void k_sort_size(int ncell, const int* need, const int* child0, const int* nblk,
                            const int* count, const int* listed, long long* sz) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= ncell) return;
  bool alias = child0[id] < 0 && nblk[id] == 1;
  sz[id] = (need[id] != 0 && !alias && count[id] > 0 && listed[id]) ? 13ll * count[id] : 0;
}

__global__ void k_sort_base(int ncell, const int* need, const int* child0, const int* nblk,
                            const int* first, const int* count, const int* listed,
                            const long long* off, long long base, long long* sbase) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= ncell) return;
  bool alias = child0[id] < 0 && nblk[id] == 1;
  if (alias) sbase[id] = 13ll * first[id];
  else if (need[id] != 0 && count[id] > 0 && listed[id]) sbase[id] = base + off[id];
  else sbase[id] = -1;
}




// ---------------------------------------------------------------- interaction lists
__global__ void k_pair_degree(int np, const int4* pairs, int* deg) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= np) return;
  atomicAdd(&deg[pairs[t].x], 1);
  atomicAdd(&deg[pairs[t].y], 1);
}

__global__ void k_pair_fill(int np, const int4* pairs, const int* off, int* cur, int* list) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= np) return;
  int a = pairs[t].x, b = pairs[t].y;
  list[off[a] + atomicAdd(&cur[a], 1)] = 2 * t;
  list[off[b] + atomicAdd(&cur[b], 1)] = 2 * t + 1;
}

__global__ void k_pair_sortlists(int ncell, const int* off, const int* deg, int* list) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= ncell) return;
  int* l = list + off[id];
  int n = deg[id];
  for (int i = 1; i < n; ++i) {
    int v = l[i], j = i - 1;
    while (j >= 0 && l[j] > v) { l[j + 1] = l[j]; --j; }
    l[j + 1] = v;
  }
}

// the other cell of the k-th pair task listed for node a, with the offset
// from a to it
__device__ __forceinline__ int pair_other(const int* alist, const int4* pairs, int v, int& ox,
                                          int& oy, int& oz, int& px, int& py, int& pz) {
  int4 tk = pairs[v >> 1];
  unpack_pair(tk.z, ox, oy, oz, px, py, pz);
  if (v & 1) {
    ox = -ox; oy = -oy; oz = -oz;
    px = -px; py = -py; pz = -pz;
    return tk.x;
  }
  return tk.y;
}

__global__ void k_block_ndt(int nblock, const int* b_leaf, const int* parent, const int* deg,
                            const int* aoff, const int* alist, const int4* pairs,
                            const int* listed, const int* ex, const int* nblk, long long* ndt) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblock) return;
  const int leaf = b_leaf[b];
  long long c = listed[leaf] ? 1 : nblk[leaf];
  for (int a = leaf; a >= 0; a = parent[a]) {
    for (int k = 0; k < deg[a]; ++k) {
      int ox, oy, oz, px, py, pz;
      const int other = pair_other(alist, pairs, alist[aoff[a] + k], ox, oy, oz, px, py, pz);
      c += ex[other];
    }
  }
  ndt[b] = c;
}

// Appends the entries a reference to node x expands to: x itself when
// listed, else the blocks of an unlisted leaf, else (depth first) those of
// its children.  Block targets are stored as -1 - block.
__device__ __forceinline__ long long emit_target(int x, int code, float4 sh, long long e,
                                                 const int* listed, const int* child0,
                                                 const int* parent, const int* count,
                                                 const int* nblk, const int* blk0,
                                                 const int* b_count, int* dt_cj, int* dt_code,
                                                 float4* dt_shift, double& cost, double wi) {
  if (count[x] == 0) return e;
  if (listed[x]) {
    dt_cj[e] = x; dt_code[e] = code; dt_shift[e] = sh;
    cost += wi * (double)min(count[x], 4096);
    return e + 1;
  }
  if (child0[x] < 0) {
    for (int k = 0; k < nblk[x]; ++k) {
      const int bj = blk0[x] + k;
      dt_cj[e] = -1 - bj; dt_code[e] = code; dt_shift[e] = sh;
      cost += wi * (double)b_count[bj];
      ++e;
    }
    return e;
  }
  // depth-first walk of the unlisted subtree: idx[l] is the next child at depth l
  int idx[32];
  int node = x, l = 0;
  idx[0] = 0;
  while (l >= 0) {
    if (idx[l] == 8) {
      --l;
      if (l >= 0) {
        node = parent[node];
        ++idx[l];
      }
      continue;
    }
    const int ch = child0[node] + idx[l];
    if (count[ch] == 0) {
      ++idx[l];
    } else if (listed[ch]) {
      dt_cj[e] = ch; dt_code[e] = code; dt_shift[e] = sh;
      cost += wi * (double)min(count[ch], 4096);
      ++e;
      ++idx[l];
    } else if (child0[ch] < 0) {
      for (int k = 0; k < nblk[ch]; ++k) {
        const int bj = blk0[ch] + k;
        dt_cj[e] = -1 - bj; dt_code[e] = code; dt_shift[e] = sh;
        cost += wi * (double)b_count[bj];
        ++e;
      }
      ++idx[l];
    } else {
      node = ch;
      idx[++l] = 0;
    }
  }
  return e;
}

__global__ void k_block_dts(int nblock, const int* b_leaf, const int* b_count, const int* parent,
                            const int* deg, const int* aoff, const int* alist, const int4* pairs,
                            const int* ntop, const int4* ijk, const int* box, const double* Ls,
                            const int* box_t, const int* ncount, const int* listed,
                            const int* child0, const int* nblk, const int* blk0,
                            const long long* dtoff, int* dt_cj, int* dt_code, float4* dt_shift,
                            unsigned long long* cost) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblock) return;
  long long e = dtoff[b];
  const int leaf = b_leaf[b];
  const double wb = (double)b_count[b];
  double c = 0;
  e = emit_target(leaf, SPH_SELF_DIR | (1 << 8), make_float4(0.f, 0.f, 0.f, 0.f), e, listed, child0,
                  parent, ncount, nblk, blk0, b_count, dt_cj, dt_code, dt_shift, c, wb);
  int bx = box[leaf];
  double L = Ls[bx];
  double et = ldexp(L, -box_t[bx]);
  int4 ta = ijk[ntop[leaf]];
  for (int a = leaf; a >= 0; a = parent[a]) {
    for (int k = 0; k < deg[a]; ++k) {
      int ox, oy, oz, px, py, pz;
      const int other = pair_other(alist, pairs, alist[aoff[a] + k], ox, oy, oz, px, py, pz);
      int oc = off_code(ox, oy, oz);
      int dir, sgn;
      if (oc > 13) { dir = oc - 14; sgn = 1; } else { dir = 12 - oc; sgn = -1; }
      int4 tb = ijk[ntop[other]];
      float sx = (float)((tb.x - ta.x) * et + px * L);
      float sy = (float)((tb.y - ta.y) * et + py * L);
      float sz = (float)((tb.z - ta.z) * et + pz * L);
      e = emit_target(other, dir | ((sgn + 1) << 8), make_float4(sx, sy, sz, 0.f), e, listed,
                      child0, parent, ncount, nblk, blk0, b_count, dt_cj, dt_code, dt_shift, c,
                      0.5 * wb);
    }
  }
  unsigned cc = c > 4.0e9 ? 0xffffffffu : (unsigned)c;
  cost[b] = (unsigned long long)(0xffffffffu - cc);  // ascending key = descending cost
}

// ---------------------------------------------------------------- work units
// A block whose sweep is long (a leaf next to a dense clump: its large-h
// particles reach 10^5 neighbours or more, so one warp would gather them
// serially for tens of milliseconds) is swept by several work units, each
// over a contiguous slice of its interaction list; the slices' partial sums
// are added, in slice order, by the unit that finishes last (see k_sweep).
// The sweep cost of a block is estimated as its chunks times the candidates
// its targets can contribute: each target's particle count (at most 4096)
// times the fraction of the target's particle box that lies within reach of
// the block's box grown by its largest h (a target wholly within reach
// contributes all its particles, a far one none).
__device__ __forceinline__ float overlap1(float lo, float hi, float a, float b) {
  const float w = hi - lo;
  const float o = fminf(hi, b) - fmaxf(lo, a);
  return w > 0.f ? fminf(fmaxf(o / w, 0.f), 1.f) : (lo >= a && lo <= b ? 1.f : 0.f);
}

// one warp per block: the lanes share the block's particles and its
// interaction entries (heavy blocks hold thousands of entries), and the
// partial sums meet in a fixed butterfly order
__global__ void k_block_cost(int nblock, const int* b_first, const int* b_count,
                             const long long* dtoff, const int* dt_cj, const float4* dt_shift,
                             const float* h, const int* pflag, const int* ncount,
                             const float4* n_lo, const float4* n_hi, const float4* b_lo,
                             const float4* b_hi, const int* nseg, unsigned long long* cost,
                             unsigned long long* total, unsigned long long* maxc) {
  const int b = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= nblock) return;
  const int f = b_first[b], bn0 = b_count[b];
  float hm = 0.f;
  int bn = 0;  // particles to sweep (pflag: only those still iterating)
  for (int k = lane; k < bn0; k += 32) {
    if (pflag && !(pflag[f + k] & 1)) continue;
    hm = fmaxf(hm, h[f + k]);
    ++bn;
  }
  bn = __reduce_add_sync(0xffffffffu, bn);
  if (bn == 0) {
    if (lane == 0) cost[b] = 0;
    return;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, o));
  const float4 l0 = b_lo[b], h0 = b_hi[b];
  double w = 0.0;
  for (long long e = dtoff[b] + lane; e < dtoff[b + 1]; e += 32) {
    const int cj = dt_cj[e];
    const float4 sh = dt_shift[e];
    int nt;
    float4 tl, th;
    if (cj >= 0) {
      nt = ncount[cj];
      tl = n_lo[cj];
      th = n_hi[cj];
    } else {
      nt = b_count[-1 - cj];
      tl = b_lo[-1 - cj];
      th = b_hi[-1 - cj];
    }
    const float fr = overlap1(tl.x + sh.x, th.x + sh.x, l0.x - hm, h0.x + hm) *
                     overlap1(tl.y + sh.y, th.y + sh.y, l0.y - hm, h0.y + hm) *
                     overlap1(tl.z + sh.z, th.z + sh.z, l0.z - hm, h0.z + hm);
    w += (double)min(nt, 4096) * fr;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  if (lane != 0) return;
  w = (w + (double)bn) * (double)((bn + 31) / 32);
  const unsigned long long c = (unsigned long long)fmin(w, 4.0e9);
  cost[b] = c;
  atomicAdd(total, c);
  // the largest unit of the present plan (its slices share the cost)
  if (maxc) atomicMax(maxc, c / (unsigned long long)max(1, nseg ? nseg[b] : 1));
}

// slices per block: the cost over four times the mean block cost, at most
// one slice per 8 interaction entries
__global__ void k_block_nseg(int nblock, const long long* dtoff, const unsigned long long* cost,
                             const unsigned long long* total, int* nseg) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblock) return;
  const double unit = 4.0 * (double)(*total) / (double)nblock + 1.0;
  const long long ent = dtoff[b + 1] - dtoff[b];
  const long long k = (long long)ceil((double)cost[b] / unit);
  nseg[b] = (int)max(1ll, min(k, ent / 8));
}

__global__ void k_block_partsz(int nblock, const int* nseg, const int* bcount, long long* psz) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblock) return;
  psz[b] = nseg[b] > 1 ? (long long)nseg[b] * bcount[b] * SPH_PART_STRIDE : 0;
}

__global__ void k_make_units(int nblock, const int* nseg, const int* uoff, const long long* dtoff,
                             const unsigned long long* cost, int* u_block, int* u_seg,
                             long long* u_e0, long long* u_e1, unsigned long long* ukey, int* uid) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblock) return;
  const int ns = nseg[b], base = uoff[b];
  const long long e0 = dtoff[b], e1 = dtoff[b + 1];
  const long long S = (e1 - e0 + ns - 1) / ns;
  const unsigned long long cu = cost[b] / (unsigned long long)ns;
  const unsigned cc = cu > 0xffffffffull ? 0xffffffffu : (unsigned)cu;
  for (int k = 0; k < ns; ++k) {
    const int u = base + k;
    u_block[u] = b;
    u_seg[u] = k;
    u_e0[u] = min(e1, e0 + k * S);
    u_e1[u] = (k == ns - 1) ? e1 : min(e1, e0 + (k + 1) * S);
    ukey[u] = (unsigned long long)(0xffffffffu - cc);  // ascending = costliest first
    uid[u] = u;
  }
}

__global__ void k_iota(int n, int* v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = i;
}


// ---------------------------------------------------------------- flat tree kernels
// Every particle carries the node that holds it at the current generation
// (pcur, -1 once its node is a leaf), so per-generation statistics are one
// pass over the particles with warp-aggregated atomics, whatever the node
// sizes (a single top cell may hold 10^5 particles of a clump).
__global__ void k_pcur_init(long long n, const unsigned long long* keys, const int* box_t,
                            const int* top_base, int K, int* pcur) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  unsigned long long key = keys[s];
  int b = (int)(key >> (3 * K));
  int t = box_t[b];
  unsigned long long tm = (key >> (3 * (K - t))) & ((1ull << (3 * t)) - 1);
  int ix = compact3(tm >> 2), iy = compact3(tm >> 1), iz = compact3(tm);
  int nb = 1 << t;
  pcur[s] = top_base[b] + (ix * nb + iy) * nb + iz;
}

__global__ void k_stats_flat(long long n, const int* pcur, const float* hs, const int4* ijk,
                             const int* box, const double* Ls, int use_h, int* acc_hmax,
                             int* acc_small) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int node = s < n ? pcur[s] : -1;
  if (__all_sync(0xffffffffu, node < 0)) return;  // every particle here sits in a leaf
  int hb = 0, small = 0;
  if (node >= 0 && use_h) {
    float hv = hs[s];
    double e = ldexp(Ls[box[node]], -ijk[node].w);
    hb = __float_as_int(hv);
    small = hv < (float)(0.5 * e) ? 1 : 0;
  }
  unsigned peers = __match_any_sync(0xffffffffu, node);
  int leader = __ffs(peers) - 1;
  // reduce within the peer group (h bits of positive floats order as ints)
  const int mx = __reduce_max_sync(peers, hb);
  const int sum = __reduce_add_sync(peers, small);
  if (lane == leader && node >= 0) {
    if (use_h) atomicMax(&acc_hmax[node], mx);
    atomicAdd(&acc_small[node], sum);
  }
}

// generation bounds live on the device: ctl[0] = first node of the
// generation, ctl[1] = one past its last node
__global__ void k_split_decide(const int* ctl, int ngmax, int split_count, float split_frac, int K,
                               const int* count, const int4* ijk, const int* acc_hmax,
                               const int* acc_small, float* hbuild, int* split) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ngmax) return;
  const int node = ctl[0] + i;
  if (node >= ctl[1]) {
    split[i] = 0;
    return;
  }
  int c = count[node];
  hbuild[node] = __int_as_float(acc_hmax[node]);
  split[i] =
      (c > split_count) && ((float)acc_small[node] > split_frac * (float)c) && (ijk[node].w < K);
}

// advance every particle to its child at the next generation (or retire it
// at its leaf) and record the children's particle ranges: a particle whose
// predecessor (successor) in Morton order lies in another child starts
// (ends) its child's range
__global__ void k_pcur_update(long long n, int* pcur, const unsigned long long* keys,
                              const int* child0, const int* first, const int* count,
                              const int4* ijk, int K, int* pnode, int* cfirst, int* cend) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  int node = pcur[s];
  if (node < 0) return;
  int c0 = child0[node];
  if (c0 < 0) {
    pnode[s] = node;
    pcur[s] = -1;
    return;
  }
  int sh = 3 * (K - ijk[node].w - 1);
  int k = (int)((keys[s] >> sh) & 7ull);
  int child = c0 + k;
  pcur[s] = child;
  long long f = first[node], e = f + count[node];
  if (s == f || (int)((keys[s - 1] >> sh) & 7ull) != k) cfirst[child] = (int)s;
  if (s == e - 1 || (int)((keys[s + 1] >> sh) & 7ull) != k) cend[child] = (int)(s + 1);
}

__global__ void k_child_counts(const int* ctl, int ngmax, const int* soff, const int* cend,
                               int* first, int* count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (ctl[2] || i >= 8 * soff[ngmax]) return;
  const int id = ctl[1] + i;
  int e = cend[id];
  count[id] = e > 0 ? e - first[id] : 0;
}

// next generation: ctl[3] is the last generation holding nodes, ctl[4 + g]
// is where generation g starts (ctl[5 + ctl[3]] where the tree ends)
__global__ void k_tree_advance(int* ctl, int ngmax, const int* soff) {
  if (ctl[2]) return;
  const int nsplit = soff[ngmax];
  if (nsplit == 0) return;
  ctl[0] = ctl[1];
  ctl[1] += 8 * nsplit;
  ctl[3] += 1;
  ctl[5 + ctl[3]] = ctl[1];
}

__global__ void k_tree_init(int* ctl, int ntop) {
  ctl[0] = 0;     // generation 0: the top cells
  ctl[1] = ntop;
  ctl[2] = 0;     // overflow
  ctl[3] = 0;     // last generation holding nodes
  ctl[4] = 0;     // generation starts
  ctl[5] = ntop;
}

__global__ void k_box_hmax(long long n, const long long* off, int nbox, const float* h, int* out) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int b = s < n ? box_of(off, nbox, s) : -1;
  int v = s < n ? __float_as_int(h[s]) : 0;
  unsigned peers = __match_any_sync(0xffffffffu, b);
  const int mx = __reduce_max_sync(peers, v);
  if (lane == __ffs(peers) - 1 && b >= 0) atomicMax(&out[b], mx);
}

// ---------------------------------------------------------------- merges
// A listed node's sorted list of a needed direction is the merge of its
// sub-lists (its children's lists, or its blocks' lists for a leaf): one CTA
// per (node, direction) ranks every element against the other sub-lists.
__device__ __forceinline__ bool mergeable(int node, const int* need, const int* child0,
                                          const int* nblk, const int* count, const int* listed) {
  return need[node] != 0 && count[node] > 0 && listed[node] && !(child0[node] < 0 && nblk[node] <= 1);
}

__global__ void k_count_positive(int n, const int* v, int* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool p = i < n && v[i] > 0;
  unsigned m = __ballot_sync(0xffffffffu, p);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(out, __popc(m));
}

__global__ void k_gather_i64(int n, const int* idx, const long long* in, long long* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[idx[i]];
}

// merge work per node: one (node, direction) segment per needed direction
// of a listed node, merged by one CTA in shared memory (k_merge_smem)
constexpr int MS_CAP = LIST_CAP;
constexpr int MS_SUB = LIST_SUB;
constexpr int MS_TPB = 256;
constexpr int MW_CAP = 512;    // largest segment merged by one warp (k_merge_warp)
constexpr int MW_WARPS = 8;
constexpr long long MW_MIN_SEGS = 65536;  // segments in a generation before small ones go to warps

__global__ void k_merge_count(int g0, int g1, const int* need, const int* child0, const int* nblk,
                              const int* count, const int* listed, long long* segs) {
  int node = g0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g1) return;
  segs[node - g0] = mergeable(node, need, child0, nblk, count, listed) ? __popc(need[node]) : 0;
}

// segment table: the node and the direction of every (node, direction)
// merge segment, so that a merge CTA finds its work without a search
__global__ void k_merge_fill(int ncell, const int* need, const int* child0, const int* nblk,
                             const int* count, const int* listed, const long long* sgo,
                             int* seg_node, unsigned char* seg_dir) {
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= ncell || !mergeable(node, need, child0, nblk, count, listed)) return;
  long long k = sgo[node];
  for (int nd = need[node]; nd; nd &= nd - 1, ++k) {
    seg_node[k] = node;
    seg_dir[k] = (unsigned char)(__ffs(nd) - 1);
  }
}

__device__ __forceinline__ int count_less_s(const float* k, const int* ix, int n, float kv, int iv) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (kv_less(k[mid], ix[mid], kv, iv)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Small segments (most of them: a leaf's few blocks, a cell of a few
// hundred particles) leave a 256-thread CTA mostly idle; there one warp
// merges one segment, MW_WARPS segments per CTA, with the same ranking:
// each element's merged position is its index in its own sub-list plus its
// rank (binary search) in every other sub-list.
__global__ void __launch_bounds__(MW_WARPS * 32)
    k_merge_warp(long long seg0, long long nseg, const int* seg_node, const unsigned char* seg_dir,
                 const int* child0, const int* count, const int* nblk, const int* blk0,
                 const int* b_first, const int* b_count, const long long* sbase, float* s_key,
                 int* s_idx) {
  __shared__ float Ks[MW_WARPS][MW_CAP];
  __shared__ int Xs[MW_WARPS][MW_CAP];
  __shared__ int sos[MW_WARPS][MS_SUB + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long sg = seg0 + (long long)blockIdx.x * MW_WARPS + w;
  if (sg >= seg0 + nseg) return;
  const int node = seg_node[sg];
  if (count[node] > MW_CAP) return;  // merged by k_merge_smem (the launch passes small_cap)
  const int d = seg_dir[sg];
  float* K = Ks[w];
  int* X = Xs[w];
  int* so = sos[w];
  const bool leaf = child0[node] < 0;
  const int nsub = leaf ? nblk[node] : 8;
  int sc = 0;
  long long base = 0;
  if (lane < nsub) {
    if (leaf) {
      const int bi = blk0[node] + lane;
      sc = b_count[bi];
      base = 13ll * b_first[bi] + (long long)d * sc;
    } else {
      const int ch = child0[node] + lane;
      sc = count[ch];
      base = sc > 0 ? sbase[ch] + (long long)d * sc : 0;
    }
  }
  int incl = sc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane < nsub) so[lane] = incl - sc;
  if (lane == nsub - 1) so[nsub] = incl;
  const long long dst0 = sbase[node] + (long long)d * count[node];
  for (int q = 0; q < nsub; ++q) {
    const int o = __shfl_sync(0xffffffffu, incl - sc, q), c = __shfl_sync(0xffffffffu, sc, q);
    const long long b = __shfl_sync(0xffffffffu, base, q);
    for (int e = lane; e < c; e += 32) {
      K[o + e] = s_key[b + e];
      X[o + e] = s_idx[b + e];
    }
  }
  __syncwarp();
  const int total = so[nsub];
  for (int e = lane; e < total; e += 32) {
    int q = 0;
    while (e >= so[q + 1]) ++q;
    const float kv = K[e];
    const int iv = X[e];
    int rank = e - so[q];
    for (int o = 0; o < nsub; ++o) {
      if (o == q) continue;
      rank += count_less_s(K + so[o], X + so[o], so[o + 1] - so[o], kv, iv);
    }
    s_key[dst0 + rank] = kv;
    s_idx[dst0 + rank] = iv;
  }
}

// one CTA per (node, direction) segment: the sub-lists (children's or the
// leaf's blocks' lists of that direction) are loaded side by side into
// shared memory and every element is ranked against the other sub-lists
__global__ void __launch_bounds__(MS_TPB)
    k_merge_smem(long long seg0, const int* seg_node, const unsigned char* seg_dir,
                 const int* child0, const int* count, const int* nblk, const int* blk0,
                 const int* b_first, const int* b_count, const long long* sbase, float* s_key,
                 int* s_idx, int small_cap) {
  __shared__ float K[MS_CAP];
  __shared__ int X[MS_CAP];
  __shared__ int so[MS_SUB + 1];
  __shared__ long long sb[MS_SUB];
  __shared__ long long dst0;
  __shared__ int nsub_s;
  {
    // segments of at most small_cap elements are merged by k_merge_warp
    const int node = seg_node[seg0 + blockIdx.x];
    if (count[node] <= small_cap) return;
  }
  if (threadIdx.x < 32) {
    // the first warp reads the sub-lists' sizes and bases in parallel and
    // scans them into offsets
    const int lane = threadIdx.x;
    const long long sg = seg0 + blockIdx.x;
    const int node = seg_node[sg];
    const int d = seg_dir[sg];
    const bool leaf = child0[node] < 0;
    const int nsub = leaf ? nblk[node] : 8;
    int sc = 0;
    long long base = 0;
    if (lane < nsub) {
      if (leaf) {
        const int bi = blk0[node] + lane;
        sc = b_count[bi];
        base = 13ll * b_first[bi] + (long long)d * sc;
      } else {
        const int ch = child0[node] + lane;
        sc = count[ch];
        base = sc > 0 ? sbase[ch] + (long long)d * sc : 0;
      }
    }
    int incl = sc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane < nsub) {
      so[lane] = incl - sc;
      sb[lane] = base;
    }
    if (lane == nsub - 1) so[nsub] = incl;
    if (lane == 0) {
      nsub_s = nsub;
      dst0 = sbase[node] + (long long)d * count[node];
    }
  }
  __syncthreads();
  const int nsub = nsub_s;
  for (int q = 0; q < nsub; ++q) {
    const int o = so[q], c = so[q + 1] - o;
    const long long b = sb[q];
    for (int e = threadIdx.x; e < c; e += MS_TPB) {
      K[o + e] = s_key[b + e];
      X[o + e] = s_idx[b + e];
    }
  }
  __syncthreads();
  const int total = so[nsub];
  for (int e = threadIdx.x; e < total; e += MS_TPB) {
    int q = 0;
    while (e >= so[q + 1]) ++q;
    const float kv = K[e];
    const int iv = X[e];
    int rank = e - so[q];
    for (int o = 0; o < nsub; ++o) {
      if (o == q) continue;
      rank += count_less_s(K + so[o], X + so[o], so[o + 1] - so[o], kv, iv);
    }
    s_key[dst0 + rank] = kv;
    s_idx[dst0 + rank] = iv;
  }
}

// ---------------------------------------------------------------- node h maxima
__global__ void k_block_hmax(int nblock, const int* b_first, const int* b_count, const float* h,
                             float* out) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= nblock) return;
  int f = b_first[warp], c = b_count[warp];
  float m = 0.f;
  for (int k = lane; k < c; k += 32) m = fmaxf(m, h[f + k]);
  m = warp_max(m);
  if (lane == 0) out[warp] = m;
}

__global__ void k_leaf_hmax(int ncell, const int* child0, const int* nblk, const int* blk0,
                            const float* bh, float* hmax) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= ncell || child0[id] >= 0) return;
  float m = 0.f;
  for (int k = 0; k < nblk[id]; ++k) m = fmaxf(m, bh[blk0[id] + k]);
  hmax[id] = m;
}

__global__ void k_internal_hmax(int g0, int g1, const int* child0, float* hmax) {
  int node = g0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g1) return;
  int c0 = child0[node];
  if (c0 < 0) return;
  float m = 0.f;
  for (int k = 0; k < 8; ++k) m = fmaxf(m, hmax[c0 + k]);
  hmax[node] = m;
}

// ---------------------------------------------------------------- bounding boxes
// of the particles (top-cell frame) of every block and node; empty nodes get
// an inverted box
__global__ void k_block_bbox(int nblock, const int* b_first, const int* b_count, const float4* pos4,
                             float4* lo, float4* hi) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= nblock) return;
  int f = b_first[warp], c = b_count[warp];
  float x0 = FLT_MAX, y0 = FLT_MAX, z0 = FLT_MAX, x1 = -FLT_MAX, y1 = -FLT_MAX, z1 = -FLT_MAX;
  for (int k = lane; k < c; k += 32) {
    const float4 p = pos4[f + k];
    x0 = fminf(x0, p.x); y0 = fminf(y0, p.y); z0 = fminf(z0, p.z);
    x1 = fmaxf(x1, p.x); y1 = fmaxf(y1, p.y); z1 = fmaxf(z1, p.z);
  }
  for (int o = 16; o > 0; o >>= 1) {
    x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
    y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, o));
    z0 = fminf(z0, __shfl_xor_sync(0xffffffffu, z0, o));
    x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
    y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    z1 = fmaxf(z1, __shfl_xor_sync(0xffffffffu, z1, o));
  }
  if (lane == 0) {
    lo[warp] = make_float4(x0, y0, z0, 0.f);
    hi[warp] = make_float4(x1, y1, z1, 0.f);
  }
}

__device__ __forceinline__ void box_union(float4& lo, float4& hi, float4 l, float4 h) {
  lo.x = fminf(lo.x, l.x); lo.y = fminf(lo.y, l.y); lo.z = fminf(lo.z, l.z);
  hi.x = fmaxf(hi.x, h.x); hi.y = fmaxf(hi.y, h.y); hi.z = fmaxf(hi.z, h.z);
}

__global__ void k_leaf_bbox(int ncell, const int* child0, const int* nblk, const int* blk0,
                            const float4* blo, const float4* bhi, float4* lo, float4* hi) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= ncell || child0[id] >= 0) return;
  float4 l = make_float4(FLT_MAX, FLT_MAX, FLT_MAX, 0.f), h = make_float4(-FLT_MAX, -FLT_MAX, -FLT_MAX, 0.f);
  for (int k = 0; k < nblk[id]; ++k) box_union(l, h, blo[blk0[id] + k], bhi[blk0[id] + k]);
  lo[id] = l;
  hi[id] = h;
}

__global__ void k_internal_bbox(int g0, int g1, const int* child0, float4* lo, float4* hi) {
  int node = g0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g1) return;
  int c0 = child0[node];
  if (c0 < 0) return;
  float4 l = make_float4(FLT_MAX, FLT_MAX, FLT_MAX, 0.f), h = make_float4(-FLT_MAX, -FLT_MAX, -FLT_MAX, 0.f);
  for (int k = 0; k < 8; ++k) box_union(l, h, lo[c0 + k], hi[c0 + k]);
  lo[node] = l;
  hi[node] = h;
}

}  // namespace

static int compute_bboxes(sph_ctx* c, cudaStream_t s) {
  SPH_TRY(dbuf_ensure(c->n_lo, sizeof(float4) * (size_t)(c->ncell + 1)));
  SPH_TRY(dbuf_ensure(c->n_hi, sizeof(float4) * (size_t)(c->ncell + 1)));
  SPH_TRY(dbuf_ensure(c->b_lo, sizeof(float4) * (size_t)(c->nblock + 1)));
  SPH_TRY(dbuf_ensure(c->b_hi, sizeof(float4) * (size_t)(c->nblock + 1)));
  { k_block_bbox<<<div_up((long long)c->nblock * 32, TPB), TPB, 0, s>>>(
      c->nblock, c->b_first.as<int>(), c->b_count.as<int>(), c->pos4.as<float4>(),
      c->b_lo.as<float4>(), c->b_hi.as<float4>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  { k_leaf_bbox<<<div_up(c->ncell, TPB), TPB, 0, s>>>(c->ncell, c->n_child0.as<int>(),
                                                     c->n_nblk.as<int>(), c->n_blk0.as<int>(),
                                                     c->b_lo.as<float4>(), c->b_hi.as<float4>(),
                                                     c->n_lo.as<float4>(), c->n_hi.as<float4>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  for (int g = (int)c->gen_start.size() - 2; g >= 0; --g) {
    int g0 = c->gen_start[g], g1 = c->gen_start[g + 1];
    if (g1 <= g0) continue;
    { k_internal_bbox<<<div_up(g1 - g0, TPB), TPB, 0, s>>>(g0, g1, c->n_child0.as<int>(),
                                                          c->n_lo.as<float4>(), c->n_hi.as<float4>()); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  return SPH_OK;
}

// ===========================================================================
// host side
// ===========================================================================
static int grow_copy(DBuf& b, size_t used, size_t want, cudaStream_t s) {
  if (b.cap >= want) return SPH_OK;
  DBuf nb;
  SPH_TRY(dbuf_ensure(nb, want));
  if (used > 0 && b.p) SPH_CUDA(cudaMemcpyAsync(nb.p, b.p, used, cudaMemcpyDeviceToDevice, s));
  SPH_CUDA(cudaStreamSynchronize(s));
  dbuf_free(b);
  b = nb;
  return SPH_OK;
}

struct NodeBufs {
  sph_ctx* c;
  int grow(size_t used_nodes, size_t want_nodes, cudaStream_t s) {
    DBuf* i4[] = {&c->n_first, &c->n_count, &c->n_parent, &c->n_child0, &c->n_top, &c->n_box};
    for (DBuf* b : i4) SPH_TRY(grow_copy(*b, used_nodes * 4, want_nodes * 4, s));
    SPH_TRY(grow_copy(c->n_ijk, used_nodes * 16, want_nodes * 16, s));
    SPH_TRY(grow_copy(c->n_hbuild, used_nodes * 4, want_nodes * 4, s));
    return SPH_OK;
  }
  NodeArrays arrays() {
    NodeArrays na;
    na.first = c->n_first.as<int>();
    na.count = c->n_count.as<int>();
    na.parent = c->n_parent.as<int>();
    na.child0 = c->n_child0.as<int>();
    na.top = c->n_top.as<int>();
    na.box = c->n_box.as<int>();
    na.ijk = c->n_ijk.as<int4>();
    na.hbuild = c->n_hbuild.as<float>();
    return na;
  }
};

template <class T>
static int d2h(T* dst, const void* src, cudaStream_t s) {
  SPH_CUDA(cudaMemcpyAsync(dst, src, sizeof(T), cudaMemcpyDeviceToHost, s));
  SPH_CUDA(cudaStreamSynchronize(s));
  return SPH_OK;
}

// Octree over the Morton-sorted particles (Section 3.2 split rule on the h
// in c->hguess).
static int build_tree(sph_ctx* c, cudaStream_t s) {
  const int n = (int)c->n;
  const int K = c->kbits;
  // top grid
  c->top_base.assign(c->nbox + 1, 0);
  for (int b = 0; b < c->nbox; ++b) {
    long long nb = 1ll << c->box_t[b];
    c->top_base[b + 1] = c->top_base[b] + (int)(nb * nb * nb);
  }
  c->ntop = c->top_base[c->nbox];
  SPH_CUDA(cudaMemcpyAsync(c->d_top_base.p, c->top_base.data(), sizeof(int) * (c->nbox + 1),
                           cudaMemcpyHostToDevice, s));
  SPH_CUDA(cudaMemcpyAsync(c->d_box_t.p, c->box_t.data(), sizeof(int) * c->nbox,
                           cudaMemcpyHostToDevice, s));
  // Node capacity: the nodes of one generation are disjoint and a node splits
  // only above split_count particles, so a generation has at most
  // max(ntop, 8 (n / (split_count + 1) + 1)) nodes; the total is kept from
  // build to build and doubled (with the tree rebuilt) if it runs out.
  // Generation bounds, counts and the overflow flag live on the device, so
  // the generations are enqueued without host round trips; the host stops
  // enqueueing once a finished generation reports that nothing split.
  const int ngmax = std::max(c->ntop, 8 * (n / (c->prm.split_count + 1) + 1));
  int mint = 64, maxt = 0;
  for (int b = 0; b < c->nbox; ++b) {
    mint = std::min(mint, c->box_t[b]);
    maxt = std::max(maxt, c->box_t[b]);
  }
  const int maxgen = K - mint + 1;
  if (c->node_cap < (size_t)c->ntop + (size_t)ngmax)
    c->node_cap = (size_t)c->ntop + 4 * (size_t)ngmax;
  SPH_TRY(dbuf_ensure(c->pnode, sizeof(int) * (size_t)n));
  SPH_TRY(dbuf_ensure(c->tmp_c, sizeof(int) * (size_t)n));  // pcur
  SPH_TRY(dbuf_ensure(c->t_cnt, sizeof(int) * ((size_t)ngmax + 1)));
  SPH_TRY(dbuf_ensure(c->t_off, sizeof(int) * ((size_t)ngmax + 1)));
  SPH_TRY(dbuf_ensure(c->tree_ctl, sizeof(int) * (size_t)(8 + maxgen + 2)));
  if (!c->tree_host) SPH_CUDA(cudaHostAlloc(&c->tree_host, 4096, cudaHostAllocDefault));
  int* pcur = c->tmp_c.as<int>();
  int* ctl = c->tree_ctl.as<int>();
  for (;;) {
    const size_t cap = c->node_cap;
    NodeBufs nbufs{c};
    SPH_TRY(nbufs.grow(0, cap, s));
    SPH_TRY(dbuf_ensure(c->n_flags, sizeof(int) * cap));
    SPH_TRY(dbuf_ensure(c->n_need, sizeof(int) * cap));
    SPH_TRY(dbuf_ensure(c->t_cnt2, sizeof(int) * cap));
    int* acc_h = c->n_flags.as<int>();  // scratch during the build: max h bits
    int* acc_s = c->n_need.as<int>();   // scratch during the build: small-h counts
    int* cend = c->t_cnt2.as<int>();
    NodeArrays na = nbufs.arrays();
    { k_init_top<<<div_up(c->ntop, TPB), TPB, 0, s>>>(c->ntop, c->d_top_base.as<int>(),
                                                    c->d_box_t.as<int>(), c->nbox,
                                                    c->keys.as<unsigned long long>(), n, K, na); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    SPH_CUDA(cudaMemsetAsync(acc_h, 0, sizeof(int) * (size_t)c->ntop, s));
    SPH_CUDA(cudaMemsetAsync(acc_s, 0, sizeof(int) * (size_t)c->ntop, s));
    { k_tree_init<<<1, 1, 0, s>>>(ctl, c->ntop); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    { k_pcur_init<<<div_up(n, TPB), TPB, 0, s>>>(n, c->keys.as<unsigned long long>(), c->d_box_t.as<int>(),
                                                c->d_top_base.as<int>(), K, pcur); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    int* hdone = reinterpret_cast<int*>(c->tree_host);
    std::vector<cudaEvent_t> evs;
    for (int g = 0; g < maxgen; ++g) {
      // stop once an earlier, finished generation reported no split
      bool done = false;
      for (int k = 0; k < (int)evs.size(); ++k)
        if (cudaEventQuery(evs[k]) == cudaSuccess && hdone[k] == 0) done = true;
      if (done) break;
      { k_stats_flat<<<div_up(n, TPB), TPB, 0, s>>>(n, pcur, c->hguess.as<float>(), na.ijk, na.box,
                                                   c->d_box_L.as<double>(), 1, acc_h, acc_s); note_launch(); }
      SPH_CUDA(cudaGetLastError());
      { k_split_decide<<<div_up(ngmax, TPB), TPB, 0, s>>>(ctl, ngmax, c->prm.split_count,
                                                         c->prm.split_frac, K, na.count, na.ijk,
                                                         acc_h, acc_s, na.hbuild, c->t_cnt.as<int>()); note_launch(); }
      SPH_CUDA(cudaGetLastError());
      SPH_TRY(scan_exclusive_i32(c->t_cnt.as<int>(), c->t_off.as<int>(), ngmax,
                                 c->t_off.as<int>() + ngmax, c->scan_tmp, s));
      { k_make_children<<<div_up(ngmax, TPB), TPB, 0, s>>>(ctl, ngmax, (int)cap, c->t_cnt.as<int>(),
                                                          c->t_off.as<int>(), na, acc_h, acc_s, cend); note_launch(); }
      SPH_CUDA(cudaGetLastError());
      { k_pcur_update<<<div_up(n, TPB), TPB, 0, s>>>(n, pcur, c->keys.as<unsigned long long>(),
                                                    na.child0, na.first, na.count, na.ijk, K,
                                                    c->pnode.as<int>(), na.first, cend); note_launch(); }
      SPH_CUDA(cudaGetLastError());
      { k_child_counts<<<div_up(ngmax, TPB), TPB, 0, s>>>(ctl, ngmax, c->t_off.as<int>(), cend,
                                                         na.first, na.count); note_launch(); }
      SPH_CUDA(cudaGetLastError());
      { k_tree_advance<<<1, 1, 0, s>>>(ctl, ngmax, c->t_off.as<int>()); note_launch(); }
      SPH_CUDA(cudaGetLastError());
      {
        cudaEvent_t e = ev_get(c);
        if (!e) return SPH_ERR_CUDA;
        SPH_CUDA(cudaMemcpyAsync(hdone + evs.size(), c->t_off.as<int>() + ngmax, sizeof(int),
                                 cudaMemcpyDeviceToHost, s));
        SPH_CUDA(cudaEventRecord(e, s));
        evs.push_back(e);
      }
    }
    int hc[8 + 64];
    SPH_CUDA(cudaMemcpyAsync(hc, ctl, sizeof(int) * (size_t)(4 + maxgen + 2), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    for (cudaEvent_t e : evs) c->ev_pool.push_back(e);
    if (hc[2]) {  // out of node capacity: double it and build again
      c->node_cap *= 2;
      continue;
    }
    const int ngen = hc[3] + 1;  // generations holding nodes
    c->gen_start.assign(hc + 4, hc + 4 + ngen + 1);
    c->ncell = hc[1];
    c->max_depth = maxt + ngen - 1;
    return SPH_OK;
  }
}

static int choose_top_levels(sph_ctx* c, cudaStream_t s) {
  // per-box max of the build h (host reduction over a D2H copy of per-box maxima)
  const int n = (int)c->n;
  std::vector<float> hmax(c->nbox, 0.f);
  SPH_TRY(dbuf_ensure(c->tmp_b, sizeof(int) * c->nbox + 64));
  SPH_CUDA(cudaMemsetAsync(c->tmp_b.p, 0, sizeof(int) * c->nbox, s));
  { k_box_hmax<<<div_up(n, TPB), TPB, 0, s>>>(n, c->d_box_off.as<long long>(), c->nbox,
                                             c->hguess.as<float>(), c->tmp_b.as<int>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_CUDA(cudaMemcpyAsync(hmax.data(), c->tmp_b.p, sizeof(float) * c->nbox, cudaMemcpyDeviceToHost, s));
  SPH_CUDA(cudaStreamSynchronize(s));
  c->box_t.assign(c->nbox, 2);
  for (int b = 0; b < c->nbox; ++b) {
    double L = c->box_L[b];
    double hm = hmax[b];
    if (!(hm > 0) || !std::isfinite(hm)) return SPH_ERR_INVALID_ARG;
    if (hm > L / 4.0) return SPH_ERR_INVALID_ARG;
    int t = (int)std::floor(std::log2(L / hm));
    while (t > 2 && L / (double)(1ll << t) < hm) --t;
    t = std::min(t, 7);
    t = std::min(t, c->kbits);
    t = std::max(t, 2);
    c->box_t[b] = t;
  }
  return SPH_OK;
}

int compute_node_hmax(sph_ctx* c, cudaStream_t s) {
  SPH_TRY(dbuf_ensure(c->n_hmax, sizeof(float) * (size_t)c->ncell));
  SPH_TRY(dbuf_ensure(c->b_hmax, sizeof(float) * (size_t)(c->nblock + 1)));
  { k_block_hmax<<<div_up((long long)c->nblock * 32, TPB), TPB, 0, s>>>(
      c->nblock, c->b_first.as<int>(), c->b_count.as<int>(), c->h.as<float>(),
      c->b_hmax.as<float>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  { k_leaf_hmax<<<div_up(c->ncell, TPB), TPB, 0, s>>>(c->ncell, c->n_child0.as<int>(),
                                                     c->n_nblk.as<int>(), c->n_blk0.as<int>(),
                                                     c->b_hmax.as<float>(), c->n_hmax.as<float>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  for (int g = (int)c->gen_start.size() - 2; g >= 0; --g) {
    int g0 = c->gen_start[g], g1 = c->gen_start[g + 1];
    if (g1 <= g0) continue;
    { k_internal_hmax<<<div_up(g1 - g0, TPB), TPB, 0, s>>>(g0, g1, c->n_child0.as<int>(),
                                                          c->n_hmax.as<float>()); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  return SPH_OK;
}

static int build_tasks(sph_ctx* c, cudaStream_t s) {
  const int ncell = c->ncell;
  // psplit flags (n_flags) cleared
  SPH_TRY(dbuf_ensure(c->n_flags, sizeof(int) * ncell));
  SPH_CUDA(cudaMemsetAsync(c->n_flags.p, 0, sizeof(int) * ncell, s));
  // Tasks of generation g join cells of octree generation g: at most one
  // self task and 13 pair tasks per cell (26 neighbours, each pair once), so
  // every buffer is sized from the octree and the generations run without a
  // host round trip; one read of the list lengths at the end.
  const int ngen = (int)c->gen_start.size() - 1;
  size_t capmax = 1;
  for (int g = 0; g < ngen; ++g)
    capmax = std::max(capmax, (size_t)14 * (size_t)(c->gen_start[g + 1] - c->gen_start[g]));
  SPH_TRY(dbuf_ensure(c->t_cur, sizeof(int4) * (capmax + 1)));
  SPH_TRY(dbuf_ensure(c->t_next, sizeof(int4) * (capmax + 1)));
  SPH_TRY(dbuf_ensure(c->t_cnt, sizeof(int) * (3 * (capmax + 1) + 1)));
  SPH_TRY(dbuf_ensure(c->t_off, sizeof(int) * (3 * (capmax + 1) + 1)));
  SPH_TRY(dbuf_ensure(c->t_final_self, sizeof(int) * ((size_t)ncell + 1)));
  SPH_TRY(dbuf_ensure(c->t_final_pair, sizeof(int4) * (13 * (size_t)ncell + 1)));
  SPH_TRY(dbuf_ensure(c->task_ctl, 64));
  int* ntp = c->task_ctl.as<int>();
  int* fin_len = ntp + 1;
  // generation 0: the top cells' self tasks and their pairs with the 13
  // half-neighbour top cells
  const int ntop = c->ntop;
  { k_top_tasks<<<div_up(ntop, TPB), TPB, 0, s>>>(ntop, c->d_top_base.as<int>(),
                                                c->d_box_t.as<int>(), c->nbox,
                                                c->n_count.as<int>(), nullptr,
                                                c->t_cnt.as<int>(), nullptr); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(scan_exclusive_i32(c->t_cnt.as<int>(), c->t_off.as<int>(), ntop,
                             c->t_off.as<int>() + ntop, c->scan_tmp, s));
  { k_top_tasks<<<div_up(ntop, TPB), TPB, 0, s>>>(ntop, c->d_top_base.as<int>(),
                                                c->d_box_t.as<int>(), c->nbox,
                                                c->n_count.as<int>(), c->t_off.as<int>(),
                                                nullptr, c->t_cur.as<int4>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_CUDA(cudaMemcpyAsync(ntp, c->t_off.as<int>() + ntop, sizeof(int), cudaMemcpyDeviceToDevice, s));
  SPH_CUDA(cudaMemsetAsync(fin_len, 0, 2 * sizeof(int), s));
  for (int g = 0; g < ngen; ++g) {
    const int cap = 14 * (c->gen_start[g + 1] - c->gen_start[g]);
    if (cap <= 0) continue;
    int* nch = c->t_cnt.as<int>();
    int* nfs = nch + (cap + 1);
    int* nfp = nfs + (cap + 1);
    int* och = c->t_off.as<int>();
    int* ofs = och + (cap + 1);
    int* ofp = ofs + (cap + 1);
    SPH_CUDA(cudaMemsetAsync(nch, 0, sizeof(int) * 3 * (size_t)(cap + 1), s));
    { k_refine<<<div_up(cap, TPB), TPB, 0, s>>>(
        ntp, cap, c->t_cur.as<int4>(), c->n_child0.as<int>(), c->n_count.as<int>(),
        c->n_hbuild.as<float>(), c->n_ijk.as<int4>(), c->n_box.as<int>(), c->d_box_L.as<double>(),
        nch, nfs, nfp, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    SPH_TRY(scan_exclusive_i32(nch, och, 3 * (cap + 1), och + 3 * (cap + 1), c->scan_tmp, s));
    { k_refine<<<div_up(cap, TPB), TPB, 0, s>>>(
        ntp, cap, c->t_cur.as<int4>(), c->n_child0.as<int>(), c->n_count.as<int>(),
        c->n_hbuild.as<float>(), c->n_ijk.as<int4>(), c->n_box.as<int>(), c->d_box_L.as<double>(),
        nullptr, nullptr, nullptr, och, ofs, ofp, c->t_next.as<int4>(), c->t_final_self.as<int>(),
        c->t_final_pair.as<int4>(), fin_len, c->n_flags.as<int>()); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    { k_refine_advance<<<1, 1, 0, s>>>(cap, och, ofs, ofp, ntp, fin_len); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    std::swap(c->t_cur, c->t_next);
  }
  int fl[3] = {0, 0, 0};
  SPH_CUDA(cudaMemcpyAsync(fl, ntp, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
  SPH_CUDA(cudaStreamSynchronize(s));
  if (fl[0] != 0) return SPH_ERR_INVALID_ARG;  // tasks left below the deepest generation
  c->nself = fl[1];
  c->npair = fl[2];
  // cell limits
  SPH_TRY(dbuf_ensure(c->n_hlim, sizeof(float) * ncell));
  for (size_t g = 0; g + 1 < c->gen_start.size(); ++g) {
    int g0 = c->gen_start[g], g1 = c->gen_start[g + 1];
    { k_hlim<<<div_up(g1 - g0, TPB), TPB, 0, s>>>(g0, g1, c->n_parent.as<int>(),
                                                c->n_flags.as<int>(), c->n_ijk.as<int4>(),
                                                c->n_box.as<int>(), c->d_box_L.as<double>(),
                                                c->n_hlim.as<float>()); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  SPH_TRY(dbuf_ensure(c->hlim, sizeof(float) * (size_t)c->n));
  { k_particle_hlim<<<div_up(c->n, TPB), TPB, 0, s>>>(c->n, c->pnode.as<int>(),
                                                    c->n_hlim.as<float>(), c->hlim.as<float>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  return SPH_OK;
}

// Work units from per-block costs (device): slices per block, unit arrays,
// partial-sum offsets, and the LPT order.  One host read of the unit and
// partial-sum counts.
static int make_plan(sph_ctx* c, const unsigned long long* bc, const unsigned long long* tot,
                     cudaStream_t s) {
  const int nblock = c->nblock;
  SPH_TRY(dbuf_ensure(c->b_nseg, sizeof(int) * (nblock + 1)));
  SPH_TRY(dbuf_ensure(c->u_off, sizeof(int) * (nblock + 1)));
  SPH_TRY(dbuf_ensure(c->b_part, sizeof(long long) * (nblock + 1)));
  SPH_TRY(dbuf_ensure(c->tmp_b, sizeof(long long) * (nblock + 1)));
  int* nseg = c->b_nseg.as<int>();
  { k_block_nseg<<<div_up(nblock, TPB), TPB, 0, s>>>(nblock, c->b_dtoff.as<long long>(), bc, tot,
                                                     nseg); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(scan_exclusive_i32(nseg, c->u_off.as<int>(), nblock, c->u_off.as<int>() + nblock,
                             c->scan_tmp, s));
  { k_block_partsz<<<div_up(nblock, TPB), TPB, 0, s>>>(nblock, nseg, c->b_count.as<int>(),
                                                       c->tmp_b.as<long long>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(scan_exclusive_i64(c->tmp_b.as<long long>(), c->b_part.as<long long>(), nblock,
                             c->b_part.as<long long>() + nblock, c->scan_tmp, s));
  int nunits = 0;
  long long npart = 0;
  SPH_TRY(d2h(&nunits, c->u_off.as<int>() + nblock, s));
  SPH_TRY(d2h(&npart, c->b_part.as<long long>() + nblock, s));
  c->nunits = nunits;
  // active-unit list of masked sweeps: tile counts, the count, the units
  SPH_TRY(dbuf_ensure(c->u_act, sizeof(int) * ((size_t)nunits + nunits / 1024 + 4)));
  SPH_TRY(dbuf_ensure(c->u_block, sizeof(int) * (nunits + 1)));
  SPH_TRY(dbuf_ensure(c->u_seg, sizeof(int) * (nunits + 1)));
  SPH_TRY(dbuf_ensure(c->u_e0, sizeof(long long) * (nunits + 1)));
  SPH_TRY(dbuf_ensure(c->u_e1, sizeof(long long) * (nunits + 1)));
  SPH_TRY(dbuf_ensure(c->u_key, sizeof(unsigned long long) * (nunits + 1) * 2));
  SPH_TRY(dbuf_ensure(c->b_order, sizeof(int) * (nunits + 1) * 2));
  SPH_TRY(dbuf_ensure(c->part, sizeof(float) * (size_t)(npart + 1)));
  c->part_cols = npart / SPH_PART_STRIDE;
  SPH_TRY(dbuf_ensure(c->blk_done, sizeof(int) * (nblock + 1)));
  SPH_CUDA(cudaMemsetAsync(c->blk_done.p, 0, sizeof(int) * (nblock + 1), s));
  unsigned long long* uk = c->u_key.as<unsigned long long>();
  int* ov = c->b_order.as<int>();
  { k_make_units<<<div_up(nblock, TPB), TPB, 0, s>>>(
      nblock, nseg, c->u_off.as<int>(), c->b_dtoff.as<long long>(), bc, c->u_block.as<int>(),
      c->u_seg.as<int>(), c->u_e0.as<long long>(), c->u_e1.as<long long>(), uk, ov); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(radix_sort_u64(uk, ov, uk + (nunits + 1), ov + (nunits + 1), nunits, 32, c->sort_tmp, s));
  ++c->build_gen;  // captured graphs hold the unit arrays and counts
  return SPH_OK;
}

// block costs of the next sweep, estimated with the current h (into the
// second half of b_cost); total and the largest unit of the present plan
static int estimate_costs(sph_ctx* c, const int* pflag, const float* h, const int* nseg,
                          cudaStream_t s) {
  const int nblock = c->nblock;
  SPH_TRY(dbuf_ensure(c->b_cost, sizeof(unsigned long long) * (nblock + 1) * 2));
  SPH_TRY(dbuf_ensure(c->plan_max, 64));
  unsigned long long* bc = c->b_cost.as<unsigned long long>() + (nblock + 1);
  unsigned long long* tot = c->plan_max.as<unsigned long long>();
  SPH_CUDA(cudaMemsetAsync(tot, 0, 2 * sizeof(unsigned long long), s));
  { k_block_cost<<<div_up((long long)nblock * 32, TPB), TPB, 0, s>>>(
      nblock, c->b_first.as<int>(), c->b_count.as<int>(), c->b_dtoff.as<long long>(),
      c->dt_cj.as<int>(), c->dt_shift.as<float4>(), h, pflag, c->n_count.as<int>(),
      c->n_lo.as<float4>(), c->n_hi.as<float4>(), c->b_lo.as<float4>(), c->b_hi.as<float4>(), nseg,
      bc, tot, tot + 1); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  return SPH_OK;
}

int replan_units(sph_ctx* c, int only_active, bool* changed, cudaStream_t s) {
  if (changed) *changed = false;
  const int nblock = c->nblock;
  if (nblock == 0) return SPH_OK;
  SPH_TRY(estimate_costs(c, only_active ? c->h_flag.as<int>() : nullptr, c->h.as<float>(),
                         c->b_nseg.as<int>(), s));
  unsigned long long host[2];
  SPH_CUDA(cudaMemcpyAsync(host, c->plan_max.p, sizeof(host), cudaMemcpyDeviceToHost, s));
  SPH_CUDA(cudaStreamSynchronize(s));
  // balanced share of one resident warp; keep the plan while its largest
  // unit stays within four such shares
  int nsm = c->sweep_grid;
  if (nsm <= 0) {  // no sweep launched yet: two CTAs per SM
    int dev = 0;
    SPH_CUDA(cudaGetDevice(&dev));
    SPH_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    nsm *= 2;
  }
  const double warps = (double)nsm * std::max(1, c->prm.warps_per_cta);
  if ((double)host[1] <= 4.0 * (double)host[0] / warps + 1.0) return SPH_OK;
  const unsigned long long* bc = c->b_cost.as<unsigned long long>() + (nblock + 1);
  SPH_TRY(make_plan(c, bc, c->plan_max.as<unsigned long long>(), s));
  if (changed) *changed = true;
  return SPH_OK;
}

static int build_blocks_and_sorts(sph_ctx* c, cudaStream_t s) {
  const int ncell = c->ncell;
  const long long n = c->n;
  // blocks
  SPH_TRY(dbuf_ensure(c->t_cnt, sizeof(int) * (ncell + 1)));
  SPH_TRY(dbuf_ensure(c->t_off, sizeof(int) * (ncell + 1)));
  SPH_TRY(dbuf_ensure(c->n_nblk, sizeof(int) * (ncell + 1)));
  SPH_TRY(dbuf_ensure(c->n_blk0, sizeof(int) * (ncell + 1)));
  int* nblk = c->n_nblk.as<int>();
  { k_leaf_nblk<<<div_up(ncell, TPB), TPB, 0, s>>>(ncell, c->n_child0.as<int>(),
                                                 c->n_count.as<int>(), c->prm.block_max, nblk); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(scan_exclusive_i32(nblk, c->t_off.as<int>(), ncell, c->t_off.as<int>() + ncell,
                             c->scan_tmp, s));
  int nblock = 0;
  SPH_TRY(d2h(&nblock, c->t_off.as<int>() + ncell, s));
  c->nblock = nblock;
  SPH_TRY(dbuf_ensure(c->b_first, sizeof(int) * (nblock + 1)));
  SPH_TRY(dbuf_ensure(c->b_count, sizeof(int) * (nblock + 1)));
  SPH_TRY(dbuf_ensure(c->b_leaf, sizeof(int) * (nblock + 1)));
  SPH_TRY(dbuf_ensure(c->n_need, sizeof(int) * (ncell + 1)));  // reused below as need
  SPH_TRY(dbuf_ensure(c->adj_off, sizeof(int) * (ncell + 1)));
  int* blk0 = c->n_blk0.as<int>();
  { k_make_blocks<<<div_up(ncell, TPB), TPB, 0, s>>>(ncell, c->n_first.as<int>(),
                                                   c->n_count.as<int>(), nblk, c->t_off.as<int>(),
                                                   c->b_first.as<int>(), c->b_count.as<int>(),
                                                   c->b_leaf.as<int>(), blk0); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  // listed nodes and expansion counts, bottom-up
  SPH_TRY(dbuf_ensure(c->n_listed, sizeof(int) * (ncell + 1)));
  SPH_TRY(dbuf_ensure(c->n_ex, sizeof(int) * (ncell + 1)));
  int* listed = c->n_listed.as<int>();
  int* nex = c->n_ex.as<int>();
  for (int g = (int)c->gen_start.size() - 2; g >= 0; --g) {
    const int g0 = c->gen_start[g], g1 = c->gen_start[g + 1];
    if (g1 <= g0) continue;
    { k_listed<<<div_up(g1 - g0, TPB), TPB, 0, s>>>(g0, g1, c->n_child0.as<int>(),
                                                   c->n_count.as<int>(), nblk, c->prm.list_cap,
                                                   listed, nex); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  // block sorts: lists of all 13 directions at [13 first, 13 (first + count))
  // needs
  int* need = c->n_need.as<int>();
  SPH_CUDA(cudaMemsetAsync(need, 0, sizeof(int) * ncell, s));
  if (c->npair > 0) {
    { k_need_pairs<<<div_up(c->npair, TPB), TPB, 0, s>>>(c->npair, c->t_final_pair.as<int4>(), need); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  { k_need_self<<<div_up(ncell, TPB), TPB, 0, s>>>(ncell, nblk, need); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  for (size_t g = 0; g + 1 < c->gen_start.size(); ++g) {
    int g0 = c->gen_start[g], g1 = c->gen_start[g + 1];
    { k_need_down<<<div_up(g1 - g0, TPB), TPB, 0, s>>>(g0, g1, c->n_child0.as<int>(), need); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  DBuf sz;
  SPH_TRY(dbuf_ensure(sz, sizeof(long long) * (ncell + 1) * 2));
  long long* szp = sz.as<long long>();
  long long* szo = szp + (ncell + 1);
  { k_sort_size<<<div_up(ncell, TPB), TPB, 0, s>>>(ncell, need, c->n_child0.as<int>(), nblk,
                                                 c->n_count.as<int>(), listed, szp); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(scan_exclusive_i64(szp, szo, ncell, szo + ncell, c->scan_tmp, s));
  long long extra = 0;
  SPH_TRY(d2h(&extra, szo + ncell, s));
  c->sorted_entries = 13ll * n + extra;
  SPH_TRY(dbuf_ensure(c->s_key, sizeof(float) * (size_t)c->sorted_entries));
  SPH_TRY(dbuf_ensure(c->s_idx, sizeof(int) * (size_t)c->sorted_entries));
  SPH_TRY(dbuf_ensure(c->n_sbase, sizeof(long long) * (ncell + 1)));
  { k_sort_base<<<div_up(ncell, TPB), TPB, 0, s>>>(ncell, need, c->n_child0.as<int>(), nblk,
                                                 c->n_first.as<int>(), c->n_count.as<int>(), listed,
                                                 szo, 13ll * n, c->n_sbase.as<long long>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  if (nblock > 0) {
    int grid = (int)std::min<long long>(div_up((long long)nblock, WS_WARPS), 152ll * 16);
    { k_sort_blocks_warp<<<grid, WS_WARPS * 32, 0, s>>>(nblock, c->b_first.as<int>(),
                                                       c->b_count.as<int>(), c->pos4.as<float4>(),
                                                       c->s_key.as<float>(), c->s_idx.as<int>()); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  SPH_TRY(build_mark(c, s, 4));
  {
    // merge segments of every cell in one scan (cells are numbered by
    // generation), one host read of the per-generation offsets, then the
    // generations from the deepest up (children before parents)
    const int ng_all = ncell;
    const int ngen = (int)c->gen_start.size();
    SPH_TRY(dbuf_ensure(sz, sizeof(long long) * (size_t)(2 * (ng_all + 1) + ngen + 2)));
    long long* sgc = sz.as<long long>();
    long long* sgo = sgc + (ng_all + 1);
    long long* gofs = sgo + (ng_all + 1);
    { k_merge_count<<<div_up(ng_all, TPB), TPB, 0, s>>>(0, ng_all, need, c->n_child0.as<int>(), nblk,
                                                       c->n_count.as<int>(), listed, sgc); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    SPH_TRY(scan_exclusive_i64(sgc, sgo, ng_all, sgo + ng_all, c->scan_tmp, s));
    SPH_TRY(dbuf_ensure(c->tmp_a, sizeof(int) * (size_t)ngen + 64));
    SPH_CUDA(cudaMemcpyAsync(c->tmp_a.p, c->gen_start.data(), sizeof(int) * ngen,
                             cudaMemcpyHostToDevice, s));
    { k_gather_i64<<<div_up(ngen, TPB), TPB, 0, s>>>(ngen, c->tmp_a.as<int>(), sgo, gofs); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    std::vector<long long> goff(ngen);
    SPH_CUDA(cudaMemcpyAsync(goff.data(), gofs, sizeof(long long) * ngen, cudaMemcpyDeviceToHost, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    const long long nseg_all = goff[ngen - 1];  // gen_start ends with the node count
    DBuf segtab;
    SPH_TRY(dbuf_ensure(segtab, (size_t)(nseg_all + 1) * 5 + 16));
    int* seg_node = segtab.as<int>();
    unsigned char* seg_dir = reinterpret_cast<unsigned char*>(seg_node + nseg_all + 1);
    { k_merge_fill<<<div_up(ng_all, TPB), TPB, 0, s>>>(ng_all, need, c->n_child0.as<int>(), nblk,
                                                       c->n_count.as<int>(), listed, sgo, seg_node,
                                                       seg_dir); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    for (int g = ngen - 2; g >= 0; --g) {
      const int g0 = c->gen_start[g], g1 = c->gen_start[g + 1];
      const long long nseg = goff[g + 1] - goff[g];
      if (g1 <= g0 || nseg <= 0) continue;
      // a generation with many segments merges its small ones one warp
      // each (more segments in flight per SM); a generation with few keeps
      // 256 threads per segment (more parallelism per segment)
      const int small_cap = nseg >= MW_MIN_SEGS ? MW_CAP : 0;
      if (small_cap > 0) {
        k_merge_warp<<<(unsigned)div_up(nseg, MW_WARPS), MW_WARPS * 32, 0, s>>>(
            goff[g], nseg, seg_node, seg_dir, c->n_child0.as<int>(), c->n_count.as<int>(), nblk,
            blk0, c->b_first.as<int>(), c->b_count.as<int>(), c->n_sbase.as<long long>(),
            c->s_key.as<float>(), c->s_idx.as<int>());
        note_launch();
      }
      { k_merge_smem<<<(unsigned)nseg, MS_TPB, 0, s>>>(
          goff[g], seg_node, seg_dir, c->n_child0.as<int>(), c->n_count.as<int>(), nblk, blk0,
          c->b_first.as<int>(), c->b_count.as<int>(), c->n_sbase.as<long long>(),
          c->s_key.as<float>(), c->s_idx.as<int>(), small_cap); note_launch(); }
      SPH_CUDA(cudaGetLastError());
    }
    SPH_CUDA(cudaStreamSynchronize(s));  // the table is freed below
    dbuf_free(segtab);
  }
  dbuf_free(sz);
  SPH_TRY(build_mark(c, s, 5));

  // ---- interaction lists per block
  int* deg = c->t_cnt.as<int>();
  int* aoff = c->adj_off.as<int>();
  SPH_CUDA(cudaMemsetAsync(deg, 0, sizeof(int) * (ncell + 1), s));
  if (c->npair > 0) {
    { k_pair_degree<<<div_up(c->npair, TPB), TPB, 0, s>>>(c->npair, c->t_final_pair.as<int4>(), deg); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  SPH_TRY(scan_exclusive_i32(deg, aoff, ncell, aoff + ncell, c->scan_tmp, s));
  SPH_TRY(dbuf_ensure(c->adj_list, sizeof(int) * (size_t)(2 * c->npair + 1)));
  SPH_TRY(dbuf_ensure(c->t_cnt2, sizeof(int) * (ncell + 1)));
  SPH_CUDA(cudaMemsetAsync(c->t_cnt2.p, 0, sizeof(int) * (ncell + 1), s));
  if (c->npair > 0) {
    { k_pair_fill<<<div_up(c->npair, TPB), TPB, 0, s>>>(c->npair, c->t_final_pair.as<int4>(), aoff,
                                                     c->t_cnt2.as<int>(), c->adj_list.as<int>()); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  { k_pair_sortlists<<<div_up(ncell, TPB), TPB, 0, s>>>(ncell, aoff, deg, c->adj_list.as<int>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(dbuf_ensure(c->b_dtoff, sizeof(long long) * (nblock + 1)));
  SPH_TRY(dbuf_ensure(c->tmp_b, sizeof(long long) * (nblock + 1)));
  { k_block_ndt<<<div_up(nblock, TPB), TPB, 0, s>>>(nblock, c->b_leaf.as<int>(),
                                                  c->n_parent.as<int>(), deg, aoff,
                                                  c->adj_list.as<int>(), c->t_final_pair.as<int4>(),
                                                  listed, nex, nblk, c->tmp_b.as<long long>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(scan_exclusive_i64(c->tmp_b.as<long long>(), c->b_dtoff.as<long long>(), nblock,
                             c->b_dtoff.as<long long>() + nblock, c->scan_tmp, s));
  long long ndt = 0;
  SPH_TRY(d2h(&ndt, c->b_dtoff.as<long long>() + nblock, s));
  c->ndt = ndt;
  SPH_TRY(dbuf_ensure(c->dt_cj, sizeof(int) * (size_t)(ndt + 1)));
  SPH_TRY(dbuf_ensure(c->dt_code, sizeof(int) * (size_t)(ndt + 1)));
  SPH_TRY(dbuf_ensure(c->dt_shift, sizeof(float4) * (size_t)(ndt + 1)));
  SPH_TRY(dbuf_ensure(c->b_cost, sizeof(unsigned long long) * (nblock + 1) * 2));
  SPH_TRY(dbuf_ensure(c->b_order, sizeof(int) * (nblock + 1) * 2));
  unsigned long long* ck = c->b_cost.as<unsigned long long>();
  { k_block_dts<<<div_up(nblock, TPB), TPB, 0, s>>>(
      nblock, c->b_leaf.as<int>(), c->b_count.as<int>(), c->n_parent.as<int>(), deg, aoff,
      c->adj_list.as<int>(), c->t_final_pair.as<int4>(), c->n_top.as<int>(), c->n_ijk.as<int4>(),
      c->n_box.as<int>(), c->d_box_L.as<double>(), c->d_box_t.as<int>(), c->n_count.as<int>(),
      listed, c->n_child0.as<int>(), nblk, blk0, c->b_dtoff.as<long long>(), c->dt_cj.as<int>(),
      c->dt_code.as<int>(), c->dt_shift.as<float4>(), ck); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  // leaves (nodes with blocks), counted on the device; read with the statistics
  SPH_TRY(dbuf_ensure(c->nleaf_dev, 64));
  SPH_CUDA(cudaMemsetAsync(c->nleaf_dev.p, 0, sizeof(int), s));
  { k_count_positive<<<div_up(ncell, TPB), TPB, 0, s>>>(ncell, nblk, c->nleaf_dev.as<int>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(build_mark(c, s, 6));
  return SPH_OK;
}

int build_mark(sph_ctx* c, cudaStream_t s, int k) {
  if (!c->profile) return SPH_OK;
  SPH_CUDA(cudaStreamSynchronize(s));
  const double t = std::chrono::duration<double, std::milli>(
                       std::chrono::steady_clock::now().time_since_epoch())
                       .count();
  if (k >= 0 && k < 8) c->prof_build_ms[k] += t - c->prof_t;
  c->prof_t = t;
  return SPH_OK;
}

int build_decomposition(sph_ctx* c, const double* pos, const float* h_guess, cudaStream_t s) {
  const long long n = c->n;
  SPH_TRY(build_mark(c, s, -1));
  const int K = c->kbits;
  int boxbits = 0;
  while ((1 << boxbits) < c->nbox) ++boxbits;
  SPH_TRY(dbuf_ensure(c->keys, 8 * (size_t)n));
  SPH_TRY(dbuf_ensure(c->keys_alt, 8 * (size_t)n));
  SPH_TRY(dbuf_ensure(c->perm, 4 * (size_t)n));
  SPH_TRY(dbuf_ensure(c->perm_alt, 4 * (size_t)n));
  SPH_TRY(dbuf_ensure(c->xs, 24 * (size_t)n));
  SPH_TRY(dbuf_ensure(c->hguess, 4 * (size_t)n));
  SPH_TRY(dbuf_ensure(c->h, 4 * (size_t)n));
  SPH_TRY(dbuf_ensure(c->pos4, 16 * (size_t)n));
  SPH_TRY(dbuf_ensure(c->p_et, 4 * (size_t)n));
  { k_keys<<<div_up(n, TPB), TPB, 0, s>>>(pos, n, c->d_box_off.as<long long>(),
                                        c->d_box_L.as<double>(), c->nbox, K,
                                        c->keys.as<unsigned long long>(), c->perm.as<int>(),
                                        c->status.as<int>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(radix_sort_u64(c->keys.as<unsigned long long>(), c->perm.as<int>(),
                         c->keys_alt.as<unsigned long long>(), c->perm_alt.as<int>(), (int)n,
                         3 * K + boxbits, c->sort_tmp, s));
  { k_gather_pos<<<div_up(n, TPB), TPB, 0, s>>>(pos, c->perm.as<int>(), n,
                                              c->d_box_off.as<long long>(),
                                              c->d_box_L.as<double>(), c->nbox, h_guess,
                                              c->xs.as<double>(), c->hguess.as<float>(),
                                              c->status.as<int>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(build_mark(c, s, 0));
  if (!h_guess) {
    // the count-only octree below a 4^3 top grid (cells split above
    // EST_SPLIT particles) gives a local-density h estimate, read off the
    // sorted keys without building that octree
    { k_h_estimate_flat<<<div_up(n, TPB), TPB, 0, s>>>(n, c->keys.as<unsigned long long>(), K, 2,
                                                     c->d_box_L.as<double>(), c->prm.n_ngb,
                                                     c->prm.h_est_mode, c->prm.h_est_factor,
                                                     c->hguess.as<float>()); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    SPH_TRY(build_mark(c, s, 1));
  }
  SPH_TRY(build_from_guess(c, s));
  if (!h_guess && c->prm.h_est_factor != 1.0f) {
    // cells were built for the widened estimate; the solve starts from the
    // estimate itself
    { k_scale<<<div_up(n, TPB), TPB, 0, s>>>(n, c->h.as<float>(), 1.0f / c->prm.h_est_factor); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  return SPH_OK;
}

int build_from_guess(sph_ctx* c, cudaStream_t s) {
  const long long n = c->n;
  ++c->build_gen;  // device-side graphs hold this decomposition's buffers
  if (c->profile) ++c->prof_builds;
  SPH_TRY(build_mark(c, s, -1));
  SPH_TRY(choose_top_levels(c, s));
  SPH_TRY(build_tree(c, s));
  { k_relpos<<<div_up(n, TPB), TPB, 0, s>>>(n, c->keys.as<unsigned long long>(), c->xs.as<double>(),
                                          c->d_box_L.as<double>(), c->d_box_t.as<int>(), c->kbits,
                                          c->pos4.as<float4>(), c->p_et.as<float>()); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  SPH_TRY(build_mark(c, s, 2));
  SPH_TRY(build_tasks(c, s));
  SPH_TRY(build_mark(c, s, 3));
  SPH_TRY(build_blocks_and_sorts(c, s));
  SPH_CUDA(cudaMemcpyAsync(c->h.p, c->hguess.p, sizeof(float) * (size_t)n,
                           cudaMemcpyDeviceToDevice, s));
  SPH_TRY(compute_node_hmax(c, s));
  SPH_TRY(compute_bboxes(c, s));
  // work units: blocks whose estimated sweep cost exceeds four times the
  // mean are cut into slices of their interaction lists; LPT order of the
  // units by estimated cost (re-planned with the current h before the
  // sweeps of the h solve and of the force when it has drifted)
  {
    SPH_TRY(estimate_costs(c, nullptr, c->hguess.as<float>(), nullptr, s));
    SPH_TRY(make_plan(c, c->b_cost.as<unsigned long long>() + (c->nblock + 1),
                      c->plan_max.as<unsigned long long>(), s));
  }
  SPH_TRY(build_mark(c, s, 7));
  return SPH_OK;
}
