// Host-side interface between the C ABI (stev_capi.cu, which owns the
// mechanism and instantiates the kernels) and the serving runtime
// (stev_server.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

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

}  // namespace host
}  // namespace stev
