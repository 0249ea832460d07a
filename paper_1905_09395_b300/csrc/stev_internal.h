// Host-side interface between the C ABI (stev_capi.cu, which owns the
// mechanism and instantiates the kernels) and the serving runtime
// (stev_server.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/stev.h"
#include "stev_layout.h"

namespace stev {
namespace host {

// Sets this thread's stev_last_error() message and returns st.
stev_status fail(stev_status st, const char* fmt, ...);
void clear_error();

// What a serving runtime needs to know about a mechanism.
struct ServeConfig {
  int device;       // CUDA device the mechanism lives on
  int S;            // species
  int ctas_per_sm;  // resident CTAs of its persistent kernel per SM
  int sms;          // SMs of the device
  int cells_per_cta;
};

// Fails (STEV_EINVAL) when the mechanism cannot serve: NULL, or thermo = MLP
// without a trained network.
stev_status serve_config(const stev_mechanism* m, ServeConfig* out);

// Launches the mechanism's persistent kernel in serving mode on `s` with
// `grid` CTAs.  ctl/slots are device pointers; mail is the device address of
// a host-mapped array of q words.
stev_status serve_launch(stev_mechanism* m, ServeCtl* ctl, ServeSlot* slots,
                         volatile long long* mail, int q, long long idle_ns, int grid,
                         cudaStream_t s);

// A mixed-precision kernel specialised for one mechanism (stev_spec.cu):
// sizes, rate-law kind, lanes per cell, DFT window (13 or 0 = run time) and
// whether it is the thermo-network kernel.
struct SpecKey {
  int S, R, Rrev, general, G, NT, net;
  bool operator==(const SpecKey& o) const {
    return S == o.S && R == o.R && Rrev == o.Rrev && general == o.general && G == o.G &&
           NT == o.NT && net == o.net;
  }
};

// Compiles the specialised kernel with NVRTC for sm_103a; the CUBIN and its
// lowered name on success, NVRTC's log in any case.  Needs no GPU.
stev_status spec_compile(const SpecKey& k, std::vector<char>* cubin, std::string* lowered,
                         std::string* log);
// Compiles and loads it into the current device's primary context.
stev_status spec_load(const SpecKey& k, cudaLibrary_t* lib, cudaKernel_t* kernel);

// Linear algebra of the Levenberg-Marquardt trainer (stev_lm.cu), device
// pointers, asynchronous on s unless stated.
// G = X X^T (n x n, full) for X [n][ldx] row-major (k columns used; ldx a
// multiple of 4, X 16-byte aligned), TF32 tensor-core products accumulated in
// FP32; *d_err (device) is set if a pipeline wait timed out.
stev_status gram_tf32(const float* X, long long n, long long k, long long ldx, float* G,
                      long long ldg, int* d_err, cudaStream_t s);
// g = X r (X as above, r 16-byte aligned).
stev_status rows_dot(const float* X, long long n, long long k, long long ldx, const float* r,
                     float* g, cudaStream_t s);
// Work arrays of damped_cg for systems of n unknowns.
struct CgWork {
  float *r, *z, *p, *q;
  double* part;
  void* state;  // the solver's scalars on the device (lm::CgState)
};
stev_status cg_work_alloc(CgWork* w, long long n);
void cg_work_free(CgWork* w);
// (A + lambda diag(A) + eps I) x = b by conjugate gradients with the Jacobi
// preconditioner, A symmetric [n][lda]; stops when the residual has fallen by
// rtol or after max_iters; *iters gets the iterations taken.  The step
// lengths are computed on the device; s is synchronised once per 16 steps.
stev_status damped_cg(const float* A, long long n, long long lda, const float* b, double lambda,
                      double eps, float* x, int max_iters, double rtol, int* iters, CgWork* w,
                      cudaStream_t s);

}  // namespace host
}  // namespace stev
