// factor.cu -- IC(0) factorisation of the (reordered) A_h on the device.
//
// Sec. 6.4: incomplete Cholesky with zero fill, L L^T = A on every position
// of the lower pattern.  Row i is computed from earlier rows k:
//   L_ik = (A_ik - sum_{j < k, j in pat(i) and pat(k)} L_ij L_kj) / L_kk,
//   L_ii = sqrt(A_ii - sum_{k < i} L_ik^2).
// In the internal numbering the rows of one DAG level are contiguous and
// independent, so each level is one launch with one warp per row.  Within a
// row the columns are taken in increasing order (each L_ik needs the L_ij,
// j < k, of the same row); the lanes share the sparse dot product with row k.
#include <cmath>

#include "gbs_device.cuh"
#include "gbs_internal.h"

namespace gbs {

namespace {

// A row of L (strict lower part) is the prefix of the same row of A.
__global__ void k_ic0_level(int r0, int r1, const int32_t* __restrict__ A_ptr,
                            const int32_t* __restrict__ A_diag, const double* __restrict__ A_val,
                            const int32_t* __restrict__ L_ptr, const int32_t* __restrict__ L_col,
                            const int32_t* __restrict__ pos, double* L_val, double* L_diag,
                            double* L_inv, int* status) {
  const int lane = threadIdx.x & 31;
  const int r = r0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (r >= r1) return;
  const int lb = L_ptr[r], le = L_ptr[r + 1];
  const int ab = A_ptr[r];
  double diag_acc = 0.0;
  for (int t = lb; t < le; ++t) {
    const int k = L_col[t];
    // sum over j < k in row k that also occur in row r (positions lb .. t-1)
    double part = 0.0;
    const int kb = L_ptr[k], ke = L_ptr[k + 1];
    for (int u = kb + lane; u < ke; u += 32) {
      const int j = L_col[u];
      int lo = lb, hi = t;  // binary search for column j among row r's first entries
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (L_col[mid] < j) lo = mid + 1;
        else hi = mid;
      }
      // entries of row r were written by lane 0 during this launch: read via L2
      if (lo < t && L_col[lo] == j) part += __ldcg(&L_val[lo]) * L_val[u];
    }
    part = warp_sum(part);
    const double lik = (A_val[ab + (t - lb)] - part) / L_diag[k];
    if (lane == 0) L_val[t] = lik;
    diag_acc += lik * lik;  // identical in every lane
    __syncwarp();
  }
  if (lane == 0) {
    const double piv = A_val[A_diag[r]] - diag_acc;
    if (!(piv > 0.0)) {
      atomicMin(&status[0], pos[r]);  // first bad row in ordering numbering
      L_diag[r] = 1.0;
      L_inv[r] = 0.0;
    } else {
      const double d = sqrt(piv);
      L_diag[r] = d;
      L_inv[r] = 1.0 / d;
    }
  }
}

__global__ void k_factor_finish(int n, int nnzL, int nnzU, const double* __restrict__ L_val,
                                const double* __restrict__ L_inv, const int32_t* __restrict__ U_map,
                                double* __restrict__ U_val, float* __restrict__ L_val32,
                                float* __restrict__ U_val32, float* __restrict__ L_inv32) {
  const int stride = gridDim.x * blockDim.x;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nnzU; t += stride) {
    const double v = L_val[U_map[t]];
    U_val[t] = v;
    U_val32[t] = (float)v;
  }
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nnzL; t += stride) L_val32[t] = (float)L_val[t];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) L_inv32[t] = (float)L_inv[t];
}

__global__ void k_sell_fill(int64_t slots, const int32_t* __restrict__ src, const double* __restrict__ csr,
                            double* __restrict__ val, float* __restrict__ val32) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < slots; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = src[t];
    const double v = k >= 0 ? csr[k] : 0.0;
    val[t] = v;
    val32[t] = (float)v;
  }
}

}  // namespace

void sell_refill(Ctx& c, Sell& S, const double* csr_val) {
  if (S.slots == 0) return;
  k_sell_fill<<<c.n_sm * 8, 256, 0, c.stream>>>(S.slots, S.src.p, csr_val, S.val.p, S.val32.p);
  GBS_CUDA(cudaGetLastError());
}

// IC(0) of the pressure mass matrix in the natural order (Sec. 6.4,
// "IC(0)-PCG(A,Q)").  Q = Q1 x Q1 [x Q1] with Q1 banded (half-bandwidth
// p - 1), so the exact Cholesky factor L1 x L1 [x L1] lies inside the lower
// pattern of Q and IC(0) reproduces it; only the band of L1 is formed:
//   L1[a][b] = (Q1[a][b] - sum_{c<b} L1[a][c] L1[b][c]) / L1[b][b]   (b < a),
//   L1[a][a] = sqrt(Q1[a][a] - sum_{c<a} L1[a][c]^2).
// One thread (m p^2 operations); *bad receives the first non-positive pivot.
__global__ void k_band_cholesky(int m, int p, const double* __restrict__ q1, double* __restrict__ l1,
                                float* __restrict__ l1_32, int* __restrict__ bad) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int a = 0; a < m; ++a) {
    for (int o = p - 1; o >= 1; --o) {  // columns b = a - o in ascending order
      const int b = a - o;
      if (b < 0) {
        l1[a * p + o] = 0.0;
        continue;
      }
      double s = q1[a * p + o];
      for (int cc = max(a - p + 1, 0); cc < b; ++cc) s -= l1[a * p + (a - cc)] * l1[b * p + (b - cc)];
      l1[a * p + o] = s / l1[b * p];
    }
    double d = q1[a * p];
    for (int cc = max(a - p + 1, 0); cc < a; ++cc) {
      const double v = l1[a * p + (a - cc)];
      d -= v * v;
    }
    if (!(d > 0.0)) {
      *bad = a;
      return;
    }
    l1[a * p] = sqrt(d);
  }
  for (int i = 0; i < m * p; ++i) l1_32[i] = (float)l1[i];
}

int64_t factor_ic0(Ctx& c) {
  if (!c.assembled) fail(GB_ERR_INVALID_ARG, "assemble before factor_ic0");
  const int n = (int)c.n_u;
  const int init = INT32_MAX;
  GBS_CUDA(cudaMemcpyAsync(c.status_d.p, &init, sizeof(int), cudaMemcpyHostToDevice, c.stream));
  for (int l = 0; l < c.nlev; ++l) {
    const int r0 = c.lev_ptr[l], r1 = c.lev_ptr[l + 1];
    const int warps = r1 - r0;
    const int block = 256;
    const int grid = (warps * 32 + block - 1) / block;
    k_ic0_level<<<grid, block, 0, c.stream>>>(r0, r1, c.A_ptr.p, c.A_diag.p, c.A_val.p, c.L_ptr.p,
                                              c.L_col.p, c.pos_d.p, c.L_val.p, c.L_diag.p, c.L_inv.p,
                                              c.status_d.p);
  }
  GBS_CUDA(cudaGetLastError());
  const int nnzL = (int)(c.nnzL - c.n_u), nnzU = nnzL;
  k_factor_finish<<<c.n_sm * 8, 256, 0, c.stream>>>(n, nnzL, nnzU, c.L_val.p, c.L_inv.p, c.U_map.p,
                                                 c.U_val.p, c.L_val32.p, c.U_val32.p, c.L_inv32.p);
  GBS_CUDA(cudaGetLastError());
  sell_refill(c, c.sL, c.L_val.p);
  sell_refill(c, c.sU, c.U_val.p);
  sell_refill(c, c.pL.data, c.L_val.p);
  sell_refill(c, c.pU.data, c.U_val.p);
  sell_refill(c, c.qL.data, c.L_val.p);
  sell_refill(c, c.qU.data, c.U_val.p);
  GBS_CUDA(cudaMemcpyAsync(c.status_d.p + 1, &init, sizeof(int), cudaMemcpyHostToDevice, c.stream));
  k_band_cholesky<<<1, 32, 0, c.stream>>>(c.N + c.p - 1, c.p, c.q1.p, c.l1.p, c.l1_32.p, c.status_d.p + 1);
  GBS_CUDA(cudaGetLastError());
  int bad = 0, bad_q = 0;
  GBS_CUDA(cudaMemcpyAsync(&bad, c.status_d.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  GBS_CUDA(cudaMemcpyAsync(&bad_q, c.status_d.p + 1, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  GBS_CUDA(cudaStreamSynchronize(c.stream));
  c.q_factored = (bad_q == INT32_MAX);
  c.ws.graph_valid = false;
  if (bad != INT32_MAX) {
    c.factored = false;
    return bad;  // row in the ordering's numbering
  }
  c.factored = true;
  return -1;
}

}  // namespace gbs
