// lattice_common.cuh -- helpers of the 2-D lattice sweep kernels (fused and resident): site
// arithmetic in the state precision and the neighbour directions of the two lattice kinds.
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

}  // namespace
}  // namespace gmrf
