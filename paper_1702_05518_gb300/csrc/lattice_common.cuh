// lattice_common.cuh -- helpers of the 2-D lattice sweep kernels (fused and resident): site
// arithmetic in the state precision, the neighbour directions of the two lattice kinds, the
// staged tile's shared-memory layout and small exact divisions.
#pragma once

#include "gmrf_device.cuh"

namespace gmrf {
namespace {

template <typename T> struct FArith;
template <> struct FArith<float> {
    // 1/P and 1/sqrt(P) within 1 ulp (P is a normal float): well inside the FP32 parity budget.
    __device__ __forceinline__ static float rcp(float x) { return rcp_approx(x); }
    __device__ __forceinline__ static float rsq(float x) { return rsqrt_approx(x); }
};
template <> struct FArith<double> {
    __device__ __forceinline__ static double rcp(double x) { return 1.0 / x; }
    __device__ __forceinline__ static double rsq(double x) { return 1.0 / sqrt(x); }
};

// Neighbour directions in a fixed order (the summation order of s_i): 8-neighbour lattice all
// (di, dj) != (0, 0) row by row; 4-neighbour lattice the four axis steps.
template <int KIND> struct Dirs;
template <> struct Dirs<kLat2D8> {
    static constexpr int N = 8;
    __device__ __forceinline__ static int di(int k) { return (k < 3) ? -1 : (k < 5 ? 0 : 1); }
    __device__ __forceinline__ static int dj(int k) { return (k < 3) ? k - 1 : (k == 3 ? -1 : (k == 4 ? 1 : k - 6)); }
    __device__ __forceinline__ static int colour(int i, int j) { return 2 * (i & 1) + (j & 1); }
};
template <> struct Dirs<kLat2D4> {
    static constexpr int N = 4;
    __device__ __forceinline__ static int di(int k) { return k == 0 ? -1 : (k == 3 ? 1 : 0); }
    __device__ __forceinline__ static int dj(int k) { return k == 1 ? -1 : (k == 2 ? 1 : 0); }
    __device__ __forceinline__ static int colour(int i, int j) { return (i + j) & 1; }
};

// Shared memory holds the staged region (natural rows gi0 .. gi0+RR-1, columns gj0 .. gj0+RC-1,
// gi0 and gj0 even) in the same colour-split layout as the state in global memory:
//   8-neighbour lattice: sub-array s = 2 (i & 1) + (j & 1), row (i - gi0) / 2, column (j - gj0) / 2;
//   4-neighbour lattice: sub-array s = (i + j) & 1,           row  i - gi0,     column (j - gj0) / 2;
// each sub-array SR x SC sites with Cp chains innermost.  A colour class is one sub-array, so a
// warp walking a class reads consecutive addresses, and staging and write-back copy rows of
// the global sub-arrays.
template <int KIND>
__device__ __forceinline__ int sm_index(int i, int j, int gi0, int gj0, int SR, int SC)
{
    if (KIND == kLat2D8) return ((2 * (i & 1) + (j & 1)) * SR + ((i - gi0) >> 1)) * SC + ((j - gj0) >> 1);
    return (((i + j) & 1) * SR + (i - gi0)) * SC + ((j - gj0) >> 1);
}

// q / d for 0 <= q < 2^16 and d >= 1 by one single-precision multiply: (q + 1/2) / d is at least
// 1/(2d) away from an integer and the two roundings err by less than 2^-7 / d, so the floor is
// exact.
__device__ __forceinline__ int div_small(int q, float rcp_d)
{
    return static_cast<int>((static_cast<float>(q) + 0.5f) * rcp_d);
}

}  // namespace
}  // namespace gmrf
