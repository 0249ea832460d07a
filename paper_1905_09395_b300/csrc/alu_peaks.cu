// Arithmetic-pipe throughput probes for the STEV roofline.
//
// The STEV step is bound by plain ALU work (FP64 pipe in the plain path, FP32
// pipe + MUFU + a small FP64 remainder in the mixed path), not by HBM, so the
// roofline denominators are per-pipe instruction rates.  Each probe runs many
// independent dependency chains per thread over a grid of (SMs x 8) blocks of
// 256 threads and reports lane-operations per second, together with the SM
// clock observed inside the kernel (clock64 against globaltimer), so that the
// rate per SM per clock can be derived.
//
// Every kernel writes exactly one value per thread into `out`, which is sized
// grid*block by the host; nothing else touches memory.
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <cuda_runtime.h>

#define CHAINS 8

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct ClockRec { unsigned long long cyc, ns; };

template <typename Op, typename T>
__global__ void probe(T seed, T b, T c, int iters, T* out, ClockRec* clk) {
  unsigned long long c0 = clock64(), t0 = gtimer();
  T a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = seed + (T)(threadIdx.x * 1e-7) + (T)(k * 1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = Op::apply(a[k], b, c);
  }
  T s = a[0];
#pragma unroll
  for (int k = 1; k < CHAINS; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) {
    clk[blockIdx.x].cyc = clock64() - c0;
    clk[blockIdx.x].ns = gtimer() - t0;
  }
}

struct DFma { static __device__ __forceinline__ double apply(double a, double b, double c) { return fma(a, b, c); } };
struct DAdd { static __device__ __forceinline__ double apply(double a, double b, double c) { return a + c; } };
struct DMul { static __device__ __forceinline__ double apply(double a, double b, double c) { return a * b; } };
struct DExp { static __device__ __forceinline__ double apply(double a, double b, double c) { return exp(-a); } };
struct DLog { static __device__ __forceinline__ double apply(double a, double b, double c) { return log(a + c); } };
struct DRcp { static __device__ __forceinline__ double apply(double a, double b, double c) { return b / a; } };
struct DMin { static __device__ __forceinline__ double apply(double a, double b, double c) { return fmin(a, b) + c; } };
// double -> float -> double round trip with an FP32 multiply in between, so
// that the compiler cannot fold the conversions away.
struct DCvt {
  static __device__ __forceinline__ double apply(double a, double b, double c) {
    return (double)((float)a * 0.99999994f);
  }
};
struct FFma { static __device__ __forceinline__ float apply(float a, float b, float c) { return fmaf(a, b, c); } };
struct FExp { static __device__ __forceinline__ float apply(float a, float b, float c) { return expf(-a); } };
struct FEx2 {
  static __device__ __forceinline__ float apply(float a, float b, float c) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-a));
    return r;
  }
};
struct FTanh {
  static __device__ __forceinline__ float apply(float a, float b, float c) {
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(a + c));
    return r;
  }
};
struct FRcp { static __device__ __forceinline__ float apply(float a, float b, float c) { return __frcp_rn(a) + c; } };

// The DFMA probe with only the first `active` lanes of each warp working (the
// others skip the loop): whether the FP64 pipe's time per warp instruction
// depends on how many lanes it carries.
__global__ void dfma_masked(double seed, double b, double c, int iters, int active, double* out) {
  double a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = seed + (double)(threadIdx.x * 1e-7) + (double)(k * 1e-3);
  if ((int)(threadIdx.x & 31) < active) {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
  }
  double s = a[0];
#pragma unroll
  for (int k = 1; k < CHAINS; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One dependent chain in one warp per SM: latency per instruction.
__global__ void dfma_latency(double seed, double b, double c, int iters, double* out, ClockRec* clk) {
  unsigned long long c0 = clock64();
  double a = seed + threadIdx.x * 1e-7;
  for (int i = 0; i < iters; ++i) a = fma(a, b, c);
  out[blockIdx.x * blockDim.x + threadIdx.x] = a;
  if (threadIdx.x == 0) { clk[blockIdx.x].cyc = clock64() - c0; clk[blockIdx.x].ns = 0; }
}

static void check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) { fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e)); exit(1); }
}

template <typename Op, typename T>
static void run(const char* name, const char* pipe, T seed, T b, T c, int iters, int sms, bool last) {
  const int block = 256, grid = sms * 8;
  T* out; ClockRec* clk;
  check(cudaMalloc(&out, sizeof(T) * grid * block), "malloc");
  check(cudaMalloc(&clk, sizeof(ClockRec) * grid), "malloc");
  probe<Op, T><<<grid, block>>>(seed, b, c, iters / 10, out, clk);  // warm-up
  check(cudaDeviceSynchronize(), "warmup");
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    probe<Op, T><<<grid, block>>>(seed, b, c, iters, out, clk);
    cudaEventRecord(e1);
    check(cudaEventSynchronize(e1), name);
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  ClockRec* h = (ClockRec*)malloc(sizeof(ClockRec) * grid);
  cudaMemcpy(h, clk, sizeof(ClockRec) * grid, cudaMemcpyDeviceToHost);
  double mhz = 0; int n = 0;
  for (int i = 0; i < grid; ++i) if (h[i].ns > 0) { mhz += (double)h[i].cyc / (double)h[i].ns * 1e3; ++n; }
  mhz /= (n ? n : 1);
  double ops = (double)grid * block * CHAINS * iters;
  double rate = ops / (best * 1e-3);
  double per_sm_clk = rate / (sms * mhz * 1e6);
  printf("  \"%s\": {\"pipe\": \"%s\", \"lane_ops_per_s\": %.6e, \"per_sm_per_clk\": %.3f, \"sm_mhz\": %.0f, \"ms\": %.3f}%s\n",
         name, pipe, rate, per_sm_clk, mhz, best, last ? "" : ",");
  free(h); cudaFree(out); cudaFree(clk);
  cudaEventDestroy(e0); cudaEventDestroy(e1);
}

int main() {
  int dev = 0; cudaDeviceProp p;
  check(cudaGetDeviceProperties(&p, dev), "props");
  const int sms = p.multiProcessorCount;
  printf("{\n  \"gpu\": \"%s\", \"sms\": %d, \"cc\": \"%d.%d\",\n", p.name, sms, p.major, p.minor);
  run<DFma, double>("dfma", "fp64", 1.0, 0.9999999, 1e-9, 4096, sms, false);
  run<DAdd, double>("dadd", "fp64", 1.0, 0.0, 1e-9, 4096, sms, false);
  run<DMul, double>("dmul", "fp64", 1.0, 0.9999999, 0.0, 4096, sms, false);
  run<DCvt, double>("cvt_f64_f32_f64_with_fmul", "conversion pair + fmul", 1.0, 0.0, 0.0, 4096, sms, false);
  run<DMin, double>("dmin_plus_dadd", "fp64", 1.0, 2.0, 1e-12, 4096, sms, false);
  run<DRcp, double>("ddiv", "fp64 (div routine)", 1.0, 1.0, 0.0, 256, sms, false);
  run<DExp, double>("dexp", "fp64 (exp routine)", 0.5, 0.0, 0.0, 256, sms, false);
  run<DLog, double>("dlog", "fp64 (log routine)", 1.5, 0.0, 1.0, 256, sms, false);
  run<FFma, float>("ffma", "fp32", 1.0f, 0.9999999f, 1e-9f, 65536, sms, false);
  run<FExp, float>("fexp", "fp32 (expf routine)", 0.5f, 0.0f, 0.0f, 16384, sms, false);
  run<FEx2, float>("ex2_approx", "mufu", 0.5f, 0.0f, 0.0f, 16384, sms, false);
  run<FTanh, float>("tanh_approx", "mufu", 0.5f, 0.0f, 0.0f, 16384, sms, false);
  run<FRcp, float>("frcp_rn", "fp32 (rcp routine)", 1.5f, 0.0f, 0.5f, 16384, sms, false);
  {
    const int block = 256, grid = sms * 8, iters = 4096;
    double* out;
    check(cudaMalloc(&out, sizeof(double) * grid * block), "malloc");
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    printf("  \"dfma_masked_warp_instr_per_sm_per_clk_at_1919mhz\": {");
    const int lanes[] = {32, 16, 8, 4, 1};
    for (int li = 0; li < 5; ++li) {
      dfma_masked<<<grid, block>>>(1.0, 0.9999999, 1e-9, iters / 10, lanes[li], out);
      check(cudaDeviceSynchronize(), "masked warmup");
      float best = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0);
        dfma_masked<<<grid, block>>>(1.0, 0.9999999, 1e-9, iters, lanes[li], out);
        cudaEventRecord(e1);
        check(cudaEventSynchronize(e1), "masked");
        float ms; cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
      }
      const double warp_instr = (double)grid * (block / 32) * CHAINS * iters;
      printf("\"%d\": %.4f%s", lanes[li], warp_instr / (best * 1e-3) / (sms * 1919e6),
             li < 4 ? ", " : "},\n");
    }
    cudaFree(out); cudaEventDestroy(e0); cudaEventDestroy(e1);
  }
  {
    double* out; ClockRec* clk;
    check(cudaMalloc(&out, sizeof(double) * sms * 32), "malloc");
    check(cudaMalloc(&clk, sizeof(ClockRec) * sms), "malloc");
    const int iters = 4096;
    dfma_latency<<<sms, 32>>>(1.0, 0.9999999, 1e-9, iters, out, clk);
    check(cudaDeviceSynchronize(), "latency");
    ClockRec h; cudaMemcpy(&h, clk, sizeof(h), cudaMemcpyDeviceToHost);
    printf("  \"dfma_dependent_latency_clk\": %.2f\n", (double)h.cyc / iters);
    cudaFree(out); cudaFree(clk);
  }
  printf("}\n");
  return 0;
}
