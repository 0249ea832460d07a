// Per-mechanism specialised kernels: the mixed-precision persistent kernels
// compiled at run time with NVRTC for one mechanism, its species, reaction and
// reversible-reaction counts and its rate-law kind as compile-time constants
// (STEV_SPEC_*, read by stev_mixed.cuh), so that the per-lane loops have known
// trip counts and the table rows sit at immediate offsets.  The source is the
// same stev_mixed.cuh the generic kernels are built from, read from the csrc
// directory beside the library; the result is loaded with cudaLibraryLoadData
// and launched like the generic kernels.
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "stev_internal.h"

namespace stev {
namespace host {

namespace {

std::string dir_of(const char* path) {
  std::string p(path ? path : "");
  const size_t k = p.rfind('/');
  return k == std::string::npos ? std::string(".") : p.substr(0, k);
}

// The csrc directory beside this library (the kernel sources).
std::string csrc_dir() {
  Dl_info info{};
  if (dladdr(reinterpret_cast<void*>(&csrc_dir), &info) && info.dli_fname)
    return dir_of(info.dli_fname) + "/csrc";
  return "csrc";
}

// CUDA's include directory (cuda_bf16.h and the NVRTC-side headers).
std::string cuda_include_dir() {
  for (const char* var : {"CUDA_HOME", "CUDA_PATH"}) {
    const char* v = std::getenv(var);
    if (v && *v) return std::string(v) + "/include";
  }
  return "/usr/local/cuda/include";
}

std::string kernel_name(const SpecKey& k) {
  char buf[96];
  if (k.net)
    std::snprintf(buf, sizeof buf, "stev::stev_mixed_net_kernel<%d, %d>", k.G, k.NT);
  else
    std::snprintf(buf, sizeof buf, "stev::stev_mixed_kernel<%d, %d>", k.G, k.NT);
  return buf;
}

}  // namespace

stev_status spec_compile(const SpecKey& k, std::vector<char>* cubin, std::string* lowered,
                         std::string* log) {
  char head[256];
  std::snprintf(head, sizeof head,
                "#define STEV_SPEC_S %d\n#define STEV_SPEC_R %d\n#define STEV_SPEC_RREV %d\n"
                "#define STEV_SPEC_GENERAL %d\n#include \"stev_mixed.cuh\"\n",
                k.S, k.R, k.Rrev, k.general);
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, head, "stev_spec.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
    return fail(STEV_ECUDA, "nvrtcCreateProgram failed");
  const std::string name = kernel_name(k);
  if (nvrtcAddNameExpression(prog, name.c_str()) != NVRTC_SUCCESS) {
    nvrtcDestroyProgram(&prog);
    return fail(STEV_ECUDA, "nvrtcAddNameExpression(%s) failed", name.c_str());
  }
  const std::string inc1 = "-I" + csrc_dir(), inc2 = "-I" + cuda_include_dir();
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device",
                        "-lineinfo", inc1.c_str(), inc2.c_str()};
  const nvrtcResult rc = nvrtcCompileProgram(prog, 6, opts);
  size_t n = 0;
  nvrtcGetProgramLogSize(prog, &n);
  std::string lg(n, '\0');
  if (n) nvrtcGetProgramLog(prog, &lg[0]);
  if (log) *log = lg;
  if (rc != NVRTC_SUCCESS) {
    nvrtcDestroyProgram(&prog);
    return fail(STEV_ECUDA, "specialised kernel (%s, S=%d R=%d): %s: %.900s", name.c_str(), k.S,
                k.R, nvrtcGetErrorString(rc), lg.c_str());
  }
  const char* low = nullptr;
  size_t cb = 0;
  if (nvrtcGetLoweredName(prog, name.c_str(), &low) != NVRTC_SUCCESS || !low ||
      nvrtcGetCUBINSize(prog, &cb) != NVRTC_SUCCESS || cb == 0) {
    nvrtcDestroyProgram(&prog);
    return fail(STEV_ECUDA, "specialised kernel %s: no lowered name or CUBIN", name.c_str());
  }
  if (lowered) *lowered = low;  // copied before the program is destroyed
  if (cubin) {
    cubin->resize(cb);
    if (nvrtcGetCUBIN(prog, cubin->data()) != NVRTC_SUCCESS) {
      nvrtcDestroyProgram(&prog);
      return fail(STEV_ECUDA, "nvrtcGetCUBIN failed for %s", name.c_str());
    }
  }
  nvrtcDestroyProgram(&prog);
  return STEV_OK;
}

stev_status spec_load(const SpecKey& k, cudaLibrary_t* lib, cudaKernel_t* kernel) {
  std::vector<char> cubin;
  std::string lowered;
  stev_status st = spec_compile(k, &cubin, &lowered, nullptr);
  if (st != STEV_OK) return st;
  cudaError_t e = cudaLibraryLoadData(lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) return fail(STEV_ECUDA, "cudaLibraryLoadData: %s", cudaGetErrorString(e));
  e = cudaLibraryGetKernel(kernel, *lib, lowered.c_str());
  if (e != cudaSuccess) {
    cudaLibraryUnload(*lib);
    *lib = nullptr;
    return fail(STEV_ECUDA, "cudaLibraryGetKernel(%s): %s", lowered.c_str(), cudaGetErrorString(e));
  }
  return STEV_OK;
}

}  // namespace host
}  // namespace stev

extern "C" stev_status stev_spec_compile_check(int n_species, int n_reactions, int n_reversible,
                                               int general, int lanes_per_cell, int dft_n,
                                               int network, char* log, size_t log_len) {
  stev::host::clear_error();
  if (n_species < 1 || n_species > 64 || n_reactions < 1 || n_reactions > 512 ||
      n_reversible < 0 || n_reversible > n_reactions)
    return stev::host::fail(STEV_EINVAL, "sizes out of range");
  if (!(lanes_per_cell == 8 || lanes_per_cell == 16 || lanes_per_cell == 32))
    return stev::host::fail(STEV_EINVAL, "lanes_per_cell must be 8, 16 or 32");
  stev::host::SpecKey k{n_species, n_reactions, n_reversible, general ? 1 : 0, lanes_per_cell,
                        dft_n == 13 ? 13 : 0, network ? 1 : 0};
  std::vector<char> cubin;
  std::string lg;
  const stev_status st = stev::host::spec_compile(k, &cubin, nullptr, &lg);
  if (log && log_len) std::snprintf(log, log_len, "%s", lg.c_str());
  return st;
}
