// Geometry shared by the build and the sweeps: Morton codes, the 13 sort
// directions of Section 3.3, and cell-pair offset encodings.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// The 26 neighbour offsets o in {-1,0,1}^3 \ {0} are coded as
// (ox+1)*9 + (oy+1)*3 + (oz+1) in [0, 27), 13 being the cell itself.
// Codes 14..26 are the 13 offsets whose first nonzero component is
// positive; sort direction d (0..12) is the unit vector of code 14 + d.
// A pair whose offset has code < 13 uses direction 12 - code with the two
// cells swapped along the axis (the "flip" of Section 3.3).
__host__ __device__ __forceinline__ int off_code(int ox, int oy, int oz) {
  return (ox + 1) * 9 + (oy + 1) * 3 + (oz + 1);
}

__host__ __device__ __forceinline__ void dir_offset(int d, int& ox, int& oy, int& oz) {
  int code = 14 + d;
  ox = code / 9 - 1;
  oy = (code / 3) % 3 - 1;
  oz = code % 3 - 1;
}

// FP32 unit vector of direction d (fixed literals so every translation
// unit rounds identically).
__host__ __device__ __forceinline__ void dir_unit(int d, float& ux, float& uy, float& uz) {
  int ox, oy, oz;
  dir_offset(d, ox, oy, oz);
  int n2 = ox * ox + oy * oy + oz * oz;
  float inv = n2 == 1 ? 1.0f : (n2 == 2 ? 0.70710677f : 0.57735026f);
  ux = ox * inv;
  uy = oy * inv;
  uz = oz * inv;
}

// sort key of a cell-relative position along direction d
__device__ __forceinline__ float sort_key(float x, float y, float z, float ux, float uy, float uz) {
  return __fmaf_rn(z, uz, __fmaf_rn(y, uy, __fmul_rn(x, ux)));
}

// 3-D Morton interleave of 21-bit coordinates, x most significant
__host__ __device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}
__host__ __device__ __forceinline__ unsigned long long morton3(unsigned x, unsigned y, unsigned z) {
  return (spread3(x) << 2) | (spread3(y) << 1) | spread3(z);
}
__host__ __device__ __forceinline__ unsigned compact3(unsigned long long v) {
  v &= 0x1249249249249249ull;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
  v = (v ^ (v >> 32)) & 0x1fffffull;
  return (unsigned)v;
}

// pair task packing: offset o (cj relative to ci, at their level) and the
// periodic image P of cj (in box lengths), each component + 1 in 2 bits
__host__ __device__ __forceinline__ int pack_pair(int ox, int oy, int oz, int px, int py, int pz) {
  return (ox + 1) | ((oy + 1) << 2) | ((oz + 1) << 4) | ((px + 1) << 6) | ((py + 1) << 8) |
         ((pz + 1) << 10);
}
__host__ __device__ __forceinline__ void unpack_pair(int c, int& ox, int& oy, int& oz, int& px,
                                                     int& py, int& pz) {
  ox = (c & 3) - 1;
  oy = ((c >> 2) & 3) - 1;
  oz = ((c >> 4) & 3) - 1;
  px = ((c >> 6) & 3) - 1;
  py = ((c >> 8) & 3) - 1;
  pz = ((c >> 10) & 3) - 1;
}
