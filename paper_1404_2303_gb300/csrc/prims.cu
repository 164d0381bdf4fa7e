// Device-wide primitives: exclusive scan and a stable LSD radix sort.
// They serve the decomposition build (Morton order, cell lists, task
// compaction); none of them is on the interaction sweeps.
#include <atomic>

#include "internal.cuh"

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launch_n(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

int dbuf_ensure(DBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return SPH_OK;
  if (b.p) {
    cudaError_t e = cudaFree(b.p);
    if (e != cudaSuccess) return SPH_ERR_CUDA;
    b.p = nullptr;
    b.cap = 0;
  }
  size_t want = bytes + bytes / 4;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    b.p = nullptr;
    return SPH_ERR_OOM;
  }
  b.cap = want;
  return SPH_OK;
}

void dbuf_free(DBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

// ---------------------------------------------------------------------------
// exclusive scan: tiles of 2048 (256 threads x 8), tile totals scanned
// recursively, then added back
// ---------------------------------------------------------------------------
namespace {
constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

template <class T>
__device__ T block_excl_scan(T v, T* sm, T* total) {
  // warp inclusive scan
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T s = lane < (SC_THREADS / 32) ? sm[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < SC_THREADS / 32) sm[lane] = s;
  }
  __syncthreads();
  T base = warp > 0 ? sm[warp - 1] : T(0);
  if (total) *total = sm[SC_THREADS / 32 - 1];
  T r = base + x - v;
  __syncthreads();
  return r;
}

template <class T>
__global__ void k_scan_tiles(const T* in, T* out, T* tile_sums, int n) {
  __shared__ T sm[32];
  int base = blockIdx.x * SC_TILE + threadIdx.x * SC_ITEMS;
  T loc[SC_ITEMS];
  T sum = 0;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    int i = base + k;
    loc[k] = i < n ? in[i] : T(0);
    sum += loc[k];
  }
  T tot;
  T pre = block_excl_scan<T>(sum, sm, &tot);
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    int i = base + k;
    if (i < n) out[i] = pre;
    pre += loc[k];
  }
  if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = tot;
}

template <class T>
__global__ void k_scan_add(T* out, const T* tile_off, int n) {
  int i = blockIdx.x * SC_TILE + threadIdx.x;
  T add = tile_off[blockIdx.x];
  for (int k = 0; k < SC_ITEMS; ++k, i += SC_THREADS)
    if (i < n) out[i] += add;
}

template <class T>
__global__ void k_scan_total(const T* in, const T* out, int n, T* total) {
  if (n > 0) *total = out[n - 1] + in[n - 1];
  else *total = 0;
}

template <class T>
int scan_rec(const T* in, T* out, int n, T* scratch, cudaStream_t s) {
  if (n <= 0) return SPH_OK;
  int nt = div_up(n, SC_TILE);
  T* sums = scratch;
  { k_scan_tiles<T><<<nt, SC_THREADS, 0, s>>>(in, out, nt > 1 ? sums : nullptr, n); note_launch(); }
  SPH_CUDA(cudaGetLastError());
  if (nt > 1) {
    T* offs = scratch + nt;
    SPH_TRY(scan_rec<T>(sums, offs, nt, scratch + 2 * nt, s));
    { k_scan_add<T><<<nt, SC_THREADS, 0, s>>>(out, offs, n); note_launch(); }
    SPH_CUDA(cudaGetLastError());
  }
  return SPH_OK;
}

template <class T>
int scan_impl(const T* in, T* out, int n, T* total, DBuf& tmp, cudaStream_t s) {
  // scratch: 2 * (n/TILE) + 2 * (n/TILE^2) + ... < 4 * n/TILE + 64
  size_t need = (size_t)(4 * (n / SC_TILE + 1) + 64) * sizeof(T);
  SPH_TRY(dbuf_ensure(tmp, need));
  SPH_TRY(scan_rec<T>(in, out, n, tmp.as<T>(), s));
  if (total) {
    if (n > 0) {
      { k_scan_total<T><<<1, 1, 0, s>>>(in, out, n, total); note_launch(); }
    } else {
      SPH_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
    }
    SPH_CUDA(cudaGetLastError());
  }
  return SPH_OK;
}
}  // namespace

int scan_exclusive_i32(const int* in, int* out, int n, int* total, DBuf& tmp, cudaStream_t s) {
  return scan_impl<int>(in, out, n, total, tmp, s);
}
int scan_exclusive_i64(const long long* in, long long* out, int n, long long* total, DBuf& tmp,
                       cudaStream_t s) {
  return scan_impl<long long>(in, out, n, total, tmp, s);
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits.  Per pass: per-tile digit histogram,
// a scan over (digit, tile), then a stable scatter that ranks each tile's
// elements round by round (256 at a time, warp match + per-warp counts).
// ---------------------------------------------------------------------------
namespace {
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;

__global__ void k_rs_hist(const unsigned long long* keys, int n, int shift, int* hist, int ntiles) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int base = blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rs_scatter(const unsigned long long* keys, const int* vals, unsigned long long* ko,
                             int* vo, int n, int shift, const int* offs, int ntiles) {
  __shared__ int wcnt[RS_THREADS / 32][257];
  __shared__ int run[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  run[threadIdx.x] = offs[threadIdx.x * ntiles + blockIdx.x];
  int base = blockIdx.x * RS_TILE;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    for (int k = threadIdx.x; k < (RS_THREADS / 32) * 257; k += RS_THREADS)
      (&wcnt[0][0])[k] = 0;
    __syncthreads();
    int i = base + r * RS_THREADS + threadIdx.x;
    bool valid = i < n;
    unsigned long long key = valid ? keys[i] : 0ull;
    int d = valid ? (int)((key >> shift) & 255) : 256;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int lrank = __popc(peers & lt);
    int leader = __ffs(peers) - 1;
    if (lane == leader) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int pos = run[d] + lrank;
      for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
      ko[pos] = key;
      vo[pos] = vals[i];
    }
    __syncthreads();
    {
      int t = 0;
      for (int w = 0; w < RS_THREADS / 32; ++w) t += wcnt[w][threadIdx.x];
      run[threadIdx.x] += t;
    }
    __syncthreads();
  }
}
}  // namespace

int radix_sort_u64(unsigned long long* keys, int* vals, unsigned long long* keys_alt, int* vals_alt,
                   int n, int nbits, DBuf& tmp, cudaStream_t s) {
  if (n <= 1) return SPH_OK;
  int ntiles = div_up(n, RS_TILE);
  int passes = (nbits + 7) / 8;
  size_t hist_bytes = (size_t)256 * ntiles * sizeof(int);
  size_t scan_scratch = (size_t)(4 * (256 * ntiles / SC_TILE + 1) + 64) * sizeof(int);
  SPH_TRY(dbuf_ensure(tmp, 2 * hist_bytes + scan_scratch + 256));
  int* hist = tmp.as<int>();
  int* offs = hist + 256 * ntiles;
  int* sscr = offs + 256 * ntiles;
  unsigned long long *ka = keys, *kb = keys_alt;
  int *va = vals, *vb = vals_alt;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    { k_rs_hist<<<ntiles, RS_THREADS, 0, s>>>(ka, n, shift, hist, ntiles); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    SPH_TRY(scan_rec<int>(hist, offs, 256 * ntiles, sscr, s));
    { k_rs_scatter<<<ntiles, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, offs, ntiles); note_launch(); }
    SPH_CUDA(cudaGetLastError());
    unsigned long long* tk = ka; ka = kb; kb = tk;
    int* tv = va; va = vb; vb = tv;
  }
  if (ka != keys) {
    SPH_CUDA(cudaMemcpyAsync(keys, ka, (size_t)n * sizeof(unsigned long long),
                             cudaMemcpyDeviceToDevice, s));
    SPH_CUDA(cudaMemcpyAsync(vals, va, (size_t)n * sizeof(int), cudaMemcpyDeviceToDevice, s));
  }
  return SPH_OK;
}
