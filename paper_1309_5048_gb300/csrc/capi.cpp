// capi.cpp -- extern "C" entry points declared in include/gbstokes.h.
// Errors inside the library are C++ exceptions of type gbs::Error; every
// entry point converts them to a status code and a thread-local message.
#include <algorithm>
#include <cstring>
#include <exception>
#include <new>
#include <string>

#include "gbs_internal.h"

namespace gbs {

namespace {
thread_local std::string g_last_error;
}

void fail(int status, const std::string& msg) { throw Error{status, msg}; }

void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    const int st = (e == cudaErrorMemoryAllocation) ? GB_ERR_OOM : GB_ERR_CUDA;
    fail(st, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

template <class T>
void DevBuf<T>::alloc(size_t count) {
  free_();
  if (count == 0) count = 1;
  void* ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(GB_ERR_OOM, "cudaMalloc failed");
  }
  p = (T*)ptr;
  n = count;
}

template <class T>
void DevBuf<T>::free_() {
  if (p) cudaFree(p);
  p = nullptr;
  n = 0;
}

template <class T>
void DevBuf<T>::upload(const T* host, size_t count, cudaStream_t s) {
  alloc(count);
  if (count) cuda_check(cudaMemcpyAsync(p, host, count * sizeof(T), cudaMemcpyHostToDevice, s), "upload");
  // pageable source: it has been staged, and may be released, when
  // cudaMemcpyAsync returns
}

template <class T>
void DevBuf<T>::zero(cudaStream_t s) {
  if (p) cuda_check(cudaMemsetAsync(p, 0, n * sizeof(T), s), "memset");
}

template struct DevBuf<int32_t>;
template struct DevBuf<double>;
template struct DevBuf<float>;

template <class F>
int guarded(F fn) {
  try {
    fn();
    return GB_OK;
  } catch (const Error& e) {
    g_last_error = e.msg;
    return e.status;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return GB_ERR_OOM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return GB_ERR_INVALID_ARG;
  }
}

void set_error(const char* msg) { g_last_error = msg; }
int bad_arg(const char* msg) {
  set_error(msg);
  return GB_ERR_INVALID_ARG;
}

// Orders the context's work stream after the caller's stream on entry and
// the caller's stream after the work stream on exit.
struct StreamOrder {
  Ctx& c;
  explicit StreamOrder(Ctx& cc) : c(cc) {
    if (c.ev_in) {
      cudaEventRecord(c.ev_in, c.user_stream);
      cudaStreamWaitEvent(c.stream, c.ev_in, 0);
    }
  }
  ~StreamOrder() {
    if (c.ev_out) {
      cudaEventRecord(c.ev_out, c.stream);
      cudaStreamWaitEvent(c.user_stream, c.ev_out, 0);
    }
  }
};

}  // namespace gbs

using namespace gbs;

struct gb_ctx {
  Ctx c;
};

extern "C" {

int gb_setup_pattern(const gb_problem* prob, void* stream, gb_ctx** out) {
  if (!prob || !out) {
    set_error("null argument");
    return GB_ERR_INVALID_ARG;
  }
  *out = nullptr;
  gb_ctx* h = nullptr;
  int st = guarded([&] {
    h = new gb_ctx();
    h->c.user_stream = (cudaStream_t)stream;
    cuda_check(cudaStreamCreateWithFlags(&h->c.stream, cudaStreamNonBlocking), "stream create");
    cuda_check(cudaEventCreateWithFlags(&h->c.ev_in, cudaEventDisableTiming), "event create");
    cuda_check(cudaEventCreateWithFlags(&h->c.ev_out, cudaEventDisableTiming), "event create");
    StreamOrder order(h->c);
    setup_pattern(h->c, *prob);
  });
  if (st != GB_OK) {
    if (h) gb_destroy(h);
    return st;
  }
  *out = h;
  return GB_OK;
}

int gb_sizes(const gb_ctx* h, int64_t* out) {
  if (!h || !out) {
    set_error("null argument");
    return GB_ERR_INVALID_ARG;
  }
  const Ctx& c = h->c;
  out[0] = c.n_u;
  out[1] = c.n_p;
  out[2] = c.nnzA;
  out[3] = c.nnzB;
  out[4] = c.nnzL;
  out[5] = c.nlev;
  out[6] = c.nrlev;
  out[7] = c.nnzQ;
  out[8] = (int64_t)held_bytes(c);
  out[9] = c.ncolours;
  return GB_OK;
}

int gb_assemble(gb_ctx* h, double nu, double cpen) {
  if (!h) return bad_arg("null context");
  return guarded([&] {
    StreamOrder order(h->c);
    assemble(h->c, nu, cpen);
  });
}

int gb_load_fourier(gb_ctx* h, int nmodes, const int32_t* kappa_host, const double* amp_host, double* f_dev) {
  if (!h) return bad_arg("null context");
  return guarded([&] {
    StreamOrder order(h->c);
    load_fourier(h->c, nmodes, kappa_host, amp_host, f_dev);
  });
}

int gb_load_manufactured(gb_ctx* h, double* f_dev) {
  if (!h) return bad_arg("null context");
  return guarded([&] {
    StreamOrder order(h->c);
    load_manufactured(h->c, f_dev);
  });
}

int gb_load_cavity(gb_ctx* h, double* f_dev) {
  if (!h) return bad_arg("null context");
  return guarded([&] {
    StreamOrder order(h->c);
    load_cavity(h->c, f_dev);
  });
}

int gb_factor_ic0(gb_ctx* h, int64_t* breakdown_row_host) {
  if (!h) return bad_arg("null context");
  int64_t row = -1;
  int st = guarded([&] {
    StreamOrder order(h->c);
    row = factor_ic0(h->c);
  });
  if (st != GB_OK) return st;
  if (breakdown_row_host) *breakdown_row_host = row;
  if (row >= 0) {
    set_error("IC(0) breakdown: non-positive pivot");
    return GB_ERR_IC0_BREAKDOWN;
  }
  return GB_OK;
}

// Status of a completed solve call, with the message for gb_last_error.
static int solve_result(int st) {
  if (st == GB_ERR_NOT_CONVERGED) set_error("a right-hand side reached max_outer (outputs written)");
  else if (st == GB_ERR_NONFINITE) set_error("a right-hand side or iterate is not finite");
  else if (st == GB_ERR_INVALID_ARG) set_error("a right-hand side violates 1^T g_p = 0 (not solved)");
  return st;
}

int gb_solve(gb_ctx* h, const double* rhs_dev, double* x_dev, int k, const gb_solve_opts* opts,
             gb_info* info_host) {
  if (!h || !opts) return bad_arg("null context or options");
  int st2 = GB_OK;
  int st = guarded([&] {
    StreamOrder order(h->c);
    st2 = solve(h->c, rhs_dev, x_dev, k, *opts, info_host, false);
  });
  return st != GB_OK ? st : solve_result(st2);
}

int gb_solve_host(gb_ctx* h, const double* rhs_host, double* x_host, int k, const gb_solve_opts* opts,
                  gb_info* info_host) {
  if (!h || !opts) return bad_arg("null context or options");
  int st2 = GB_OK;
  int st = guarded([&] {
    StreamOrder order(h->c);
    st2 = solve_host(h->c, rhs_host, x_host, k, *opts, info_host);
  });
  return st != GB_OK ? st : solve_result(st2);
}

int gb_solve_adjoint(gb_ctx* h, const double* grad_dev, double* lam_dev, int k, const gb_solve_opts* opts,
                     gb_info* info_host) {
  if (!h || !opts) return bad_arg("null context or options");
  int st2 = GB_OK;
  int st = guarded([&] {
    StreamOrder order(h->c);
    st2 = solve(h->c, grad_dev, lam_dev, k, *opts, info_host, true);
  });
  return st != GB_OK ? st : solve_result(st2);
}

int gb_dnu(gb_ctx* h, const double* lam_dev, const double* x_dev, int k, double* out_host) {
  if (!h) return bad_arg("null context");
  return guarded([&] {
    StreamOrder order(h->c);
    dnu(h->c, lam_dev, x_dev, k, out_host);
  });
}

int gb_set_kernel_variants(gb_ctx* h, int precision, int spmv, int trsv) {
  if (!h) return bad_arg("null context");
  if (precision < 0 || precision > 1 || spmv < -1 || spmv > 3 || trsv < -1 || trsv > 18) {
    set_error("bad kernel variant request");
    return GB_ERR_INVALID_ARG;
  }
  if (!gbs::trsv_available(h->c, trsv)) {
    set_error("sweep layout unavailable: a row of the IC(0) factor does not fit one block");
    return GB_ERR_INVALID_ARG;
  }
  h->c.var_spmv[precision] = spmv;
  h->c.var_trsv[precision] = trsv;
  h->c.ws.graph_valid = false;
  return GB_OK;
}

int gb_set_batch_sweep(gb_ctx* h, int precision, int width, int variant) {
  if (!h) return bad_arg("null context");
  if (precision < 0 || precision > 1 || (width != 8 && width != 32) || variant < -1 || variant > 1) {
    set_error("bad batch sweep request");
    return GB_ERR_INVALID_ARG;
  }
  h->c.var_trsv_batch[precision][width == 8 ? 0 : 1] = variant;
  h->c.ws.graph_valid = false;
  return GB_OK;
}

int gb_get_batch_sweep(const gb_ctx* h, int precision, int width, int* variant) {
  if (!h) return bad_arg("null context");
  if (precision < 0 || precision > 1 || (width != 8 && width != 32) || !variant) {
    set_error("bad batch sweep query");
    return GB_ERR_INVALID_ARG;
  }
  *variant = h->c.var_trsv_batch[precision][width == 8 ? 0 : 1];
  return GB_OK;
}

int gb_get_kernel_variants(const gb_ctx* h, int precision, int* spmv, int* trsv) {
  if (!h) return bad_arg("null context");
  if (precision < 0 || precision > 1 || !spmv || !trsv) {
    set_error("bad kernel variant query");
    return GB_ERR_INVALID_ARG;
  }
  *spmv = h->c.var_spmv[precision];
  *trsv = h->c.var_trsv[precision];
  return GB_OK;
}

int gb_lanczos(gb_ctx* h, int rhs, double* delta_host, double* gamma_host, int cap, int* count) {
  if (!h || !count) return bad_arg("null context or count");
  return guarded([&] {
    StreamOrder order(h->c);
    *count = lanczos_coeffs(h->c, rhs, delta_host, gamma_host, cap);
  });
}

int gb_ritz_extremes(gb_ctx* h, int rhs, int exclude_one, double* out_host) {
  if (!h || !out_host) return bad_arg("null context or output");
  return guarded([&] {
    StreamOrder order(h->c);
    ritz_extremes(h->c, rhs, exclude_one, out_host);
  });
}

int gb_time_kernel(gb_ctx* h, int which, int reps, double* ms_host) {
  if (!h || !ms_host) return bad_arg("null context or output");
  return guarded([&] {
    StreamOrder order(h->c);
    *ms_host = time_kernel(h->c, which, reps);
  });
}

int gb_dnu_noalloc(gb_ctx* h, const double* lam_dev, const double* x_dev, int k, double* out_host) {
  if (!h) return bad_arg("null context");
  return guarded([&] {
    StreamOrder order(h->c);
    dnu_noalloc(h->c, lam_dev, x_dev, k, out_host);
  });
}

int gb_apply(gb_ctx* h, int which, const double* x_dev, double* y_dev) {
  if (!h) return bad_arg("null context");
  return guarded([&] {
    StreamOrder order(h->c);
    apply_operator(h->c, which, x_dev, y_dev);
  });
}

int gb_export(gb_ctx* h, int what, void* p0, void* p1, void* p2) {
  if (!h) return bad_arg("null context");
  return guarded([&] {
    Ctx& c = h->c;
    StreamOrder order(c);
    const int64_t n = c.n_u;
    auto dl = [&](void* dst, const void* src, size_t bytes) {
      cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c.stream), "export");
    };
    if (what == 0 || what == 1) {
      // natural numbering; rows re-sorted by column
      const bool isA = what == 0;
      const int64_t nrows = isA ? n : c.n_p;
      const std::vector<int32_t>& ptr = isA ? c.hA_ptr : c.hB_ptr;
      const std::vector<int32_t>& col = isA ? c.hA_col : c.hB_col;
      std::vector<double> val(col.size());
      dl(val.data(), isA ? c.A_val.p : c.B_val.p, sizeof(double) * col.size());
      cuda_check(cudaStreamSynchronize(c.stream), "export sync");
      std::vector<int32_t> iord(n);
      for (int64_t r = 0; r < n; ++r) iord[r] = c.order[r];
      int64_t* optr = (int64_t*)p0;
      int32_t* ocol = (int32_t*)p1;
      double* oval = (double*)p2;
      std::vector<int64_t> start(nrows + 1, 0);
      for (int64_t r = 0; r < nrows; ++r) {
        const int64_t nat = isA ? c.order[r] : r;
        start[nat + 1] = ptr[r + 1] - ptr[r];
      }
      for (int64_t r = 0; r < nrows; ++r) start[r + 1] += start[r];
      if (optr) std::copy(start.begin(), start.end(), optr);
      std::vector<std::pair<int32_t, double>> row;
      for (int64_t r = 0; r < nrows; ++r) {
        const int64_t nat = isA ? c.order[r] : r;
        row.clear();
        for (int32_t t = ptr[r]; t < ptr[r + 1]; ++t) row.emplace_back(iord[col[t]], val[t]);
        std::sort(row.begin(), row.end());
        for (size_t u = 0; u < row.size(); ++u) {
          if (ocol) ocol[start[nat] + u] = row[u].first;
          if (oval) oval[start[nat] + u] = row[u].second;
        }
      }
    } else if (what == 2) {
      // factor in the ordering's numbering: row i = internal row of position i
      std::vector<int32_t> Lptr(n + 1), Lcol(c.nnzL - n);
      std::vector<double> Lval(c.nnzL - n), Ldiag(n);
      dl(Lptr.data(), c.L_ptr.p, sizeof(int32_t) * (n + 1));
      if (c.nnzL > n) {
        dl(Lcol.data(), c.L_col.p, sizeof(int32_t) * (c.nnzL - n));
        dl(Lval.data(), c.L_val.p, sizeof(double) * (c.nnzL - n));
      }
      dl(Ldiag.data(), c.L_diag.p, sizeof(double) * n);
      cuda_check(cudaStreamSynchronize(c.stream), "export sync");
      std::vector<int32_t> pos_to_int(n);
      for (int64_t r = 0; r < n; ++r) pos_to_int[c.int_to_pos[r]] = (int32_t)r;
      int64_t* optr = (int64_t*)p0;
      int32_t* ocol = (int32_t*)p1;
      double* oval = (double*)p2;
      int64_t off = 0;
      std::vector<std::pair<int32_t, double>> row;
      for (int64_t i = 0; i < n; ++i) {
        const int32_t r = pos_to_int[i];
        row.clear();
        for (int32_t t = Lptr[r]; t < Lptr[r + 1]; ++t) row.emplace_back(c.int_to_pos[Lcol[t]], Lval[t]);
        std::sort(row.begin(), row.end());
        row.emplace_back((int32_t)i, Ldiag[r]);
        if (optr) optr[i] = off;
        for (auto& e : row) {
          if (ocol) ocol[off] = e.first;
          if (oval) oval[off] = e.second;
          ++off;
        }
      }
      if (optr) optr[n] = off;
    } else if (what == 3) {
      if (p0) std::memcpy(p0, c.perm.data(), sizeof(int32_t) * n);
      if (p1) std::memcpy(p1, c.level.data(), sizeof(int32_t) * n);
      if (p2) std::memcpy(p2, c.rlevel.data(), sizeof(int32_t) * n);
    } else if (what == 4) {
      if (p1) dl(p1, c.wmean.p, sizeof(double) * c.n_p);
      if (p2) dl(p2, c.Qdiag.p, sizeof(double) * c.n_p);
      cuda_check(cudaStreamSynchronize(c.stream), "export sync");
    } else if (what == 5) {
      if (p0) dl(p0, c.Q_ptr.p, sizeof(int32_t) * (c.n_p + 1));
      if (p1) dl(p1, c.Q_col.p, sizeof(int32_t) * c.nnzQ);
      if (p2) dl(p2, c.Q_val.p, sizeof(double) * c.nnzQ);
      cuda_check(cudaStreamSynchronize(c.stream), "export sync");
    } else if (what == 6) {
      if (!c.q_factored) fail(GB_ERR_INVALID_ARG, "factor_ic0 must succeed before exporting the factor of Q");
      const size_t band = (size_t)(c.N + c.p - 1) * c.p;
      if (p0) dl(p0, c.q1.p, sizeof(double) * band);
      if (p1) dl(p1, c.l1.p, sizeof(double) * band);
      cuda_check(cudaStreamSynchronize(c.stream), "export sync");
    } else {
      fail(GB_ERR_INVALID_ARG, "unknown export");
    }
  });
}

void gb_destroy(gb_ctx* h) {
  if (!h) return;
  try {
    if (h->c.stream) cudaStreamSynchronize(h->c.stream);
    release_workspace(h->c);
  } catch (...) {
  }
  cudaStream_t s = h->c.stream;
  cudaEvent_t e1 = h->c.ev_in, e2 = h->c.ev_out;
  delete h;  // device buffers are released by their destructors
  if (e1) cudaEventDestroy(e1);
  if (e2) cudaEventDestroy(e2);
  if (s) cudaStreamDestroy(s);
}

const char* gb_status_string(int s) {
  switch (s) {
    case GB_OK: return "ok";
    case GB_ERR_INVALID_ARG: return "invalid argument";
    case GB_ERR_CUDA: return "CUDA error";
    case GB_ERR_OOM: return "out of memory";
    case GB_ERR_IC0_BREAKDOWN: return "IC(0) breakdown";
    case GB_ERR_NOT_CONVERGED: return "not converged";
    case GB_ERR_NONFINITE: return "non-finite value";
    case GB_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* gb_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
