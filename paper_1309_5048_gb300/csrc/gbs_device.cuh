// gbs_device.cuh -- device helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace gbs {

constexpr int kBlock = 256;  // threads per block for vector kernels

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Mask of the G consecutive lanes (G a power of two <= 32) holding this lane.
// Shuffles restricted to it stay valid when other groups of the same warp
// have left a loop or returned.
template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (G == 32) {
    return 0xffffffffu;
  } else {
    return ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
  }
}

// Sum over the lane's group of G consecutive lanes.
template <int G>
__device__ __forceinline__ double group_sum(double v) {
  const unsigned m = group_mask<G>();
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
  return v;
}

template <int G>
__device__ __forceinline__ float group_sumf(float v) {
  const unsigned m = group_mask<G>();
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
  return v;
}

// Block-wide reduction of NS sums per RHS slot.  Each thread holds vals for
// its own RHS slot `slot` (0..K-1); K divides 32.  The per-block results are
// written to partial[(blockIdx.x * K + slot) * NS + s].  Lanes of a warp that
// share a slot are summed with shuffles in a fixed pattern, then warps are
// summed in warp order by thread 0..K-1: deterministic for a fixed launch.
template <int K, int NS>
__device__ __forceinline__ void block_partials(const double (&vals)[NS], double* partial) {
  __shared__ double sh[kBlock / 32][32][NS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // a previous call's readers are done with sh
  double v[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    v[s] = vals[s];
    // lanes l and l + K*m share a slot
#pragma unroll
    for (int o = 16; o >= K; o >>= 1) v[s] += __shfl_xor_sync(0xffffffffu, v[s], o);
  }
  if (lane < K) {
#pragma unroll
    for (int s = 0; s < NS; ++s) sh[warp][lane][s] = v[s];
  }
  __syncthreads();
  if (threadIdx.x < K) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double acc = 0.0;
      for (int w = 0; w < nw; ++w) acc += sh[w][threadIdx.x][s];
      partial[((size_t)blockIdx.x * K + threadIdx.x) * NS + s] = acc;
    }
  }
}

// Returns true in exactly one block: the last to finish.  That block then
// sees all partials (after the fence) and must reset *counter to 0.
__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// Inside the last block: total[slot*NS+s] = sum over blocks of partials, in
// a fixed order.  Each of the K*NS sums gets TPS consecutive threads (a
// power of two <= 32); each thread adds a fixed strided subset of the blocks,
// then the TPS threads combine with a fixed shuffle tree.
template <int K, int NS>
__device__ __forceinline__ void finalize_partials(const double* partial, int nblocks, double* total) {
  constexpr int NSUM = K * NS;
  constexpr int TPS = (kBlock / NSUM >= 32) ? 32 : (kBlock / NSUM >= 16 ? 16 : (kBlock / NSUM >= 8 ? 8 : (kBlock / NSUM >= 4 ? 4 : (kBlock / NSUM >= 2 ? 2 : 1))));
  static_assert(NSUM * TPS <= kBlock, "too many sums for one block");
  const int idx = threadIdx.x / TPS, sub = threadIdx.x % TPS;
  double acc = 0.0;
  if (idx < NSUM)
    for (int b = sub; b < nblocks; b += TPS) acc += partial[(size_t)b * NSUM + idx];
  acc = group_sum<TPS>(acc);
  if (sub == 0 && idx < NSUM) total[idx] = acc;
  __syncthreads();
}

// Knot xi_j of the uniform open knot vector of degree q with N elements.
__device__ __forceinline__ double open_knot(int j, int q, int N) {
  int t = j - q;
  t = t < 0 ? 0 : (t > N ? N : t);
  return (double)t / (double)N;
}

// Values and first derivatives of the q+1 B-splines of degree q that are
// nonzero on element e (function indices e..e+q), at x in that element, from
// the Cox-de Boor recursion (Sec. 2.1).  q <= 6.
__device__ inline void bspline_element(int N, int q, int e, double x, double* val, double* der) {
  // bas[t] holds B_{e+t-r, r} during step r (t = r..q index the live ones)
  double bas[8];
  for (int t = 0; t <= q; ++t) bas[t] = 0.0;
  bas[q] = 1.0;  // B_{e+q, 0}: the knot span of element e is [xi_{e+q}, xi_{e+q+1})
  double lower[8];  // degree q-1 values kept for the derivative
  for (int r = 1; r <= q; ++r) {
    if (r == q)
      for (int t = 0; t <= q; ++t) lower[t] = bas[t];
    // new B_{i,r} for i = e+q-r .. e+q, stored at slot t = i - e
    double nb[8];
    for (int t = 0; t <= q; ++t) nb[t] = 0.0;
    for (int t = q - r; t <= q; ++t) {
      const int i = e + t;
      const double a0 = open_knot(i, q, N), a1 = open_knot(i + r, q, N);
      const double b0 = open_knot(i + 1, q, N), b1 = open_knot(i + r + 1, q, N);
      double v = 0.0;
      if (a1 > a0) v += (x - a0) / (a1 - a0) * bas[t];
      if (t + 1 <= q && b1 > b0) v += (b1 - x) / (b1 - b0) * bas[t + 1];
      nb[t] = v;
    }
    for (int t = 0; t <= q; ++t) bas[t] = nb[t];
  }
  if (q == 0) {
    val[0] = 1.0;
    der[0] = 0.0;
    return;
  }
  for (int t = 0; t <= q; ++t) {
    const int i = e + t;
    val[t] = bas[t];
    double d = 0.0;
    const double a0 = open_knot(i, q, N), a1 = open_knot(i + q, q, N);
    const double b0 = open_knot(i + 1, q, N), b1 = open_knot(i + q + 1, q, N);
    if (a1 > a0) d += q / (a1 - a0) * lower[t];
    if (t + 1 <= q && b1 > b0) d -= q / (b1 - b0) * lower[t + 1];
    der[t] = d;
  }
}

}  // namespace gbs
