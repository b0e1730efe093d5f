// cr_probe.cu -- throughput probes of the units the cRKFR kernels use.
//
// The measured peaks cover HBM copy and BF16 tensor throughput only; the
// pair fluxes run on the FP32 FMA pipe and the MUFU unit, the state update on
// the FP64 pipe (which on this GPU also executes float <-> double
// conversions).  Each probe runs independent operation chains on every SM
// (8 chains per thread, 256 threads per CTA, 8 CTAs per SM) and is timed with
// CUDA events; results are lane-operations per second (HBM: bytes/s read+write).
#include <cuda_runtime.h>

#include "../../include/cr.h"
#include "crkfr_physics.cuh"

namespace {

constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) p_ffma(float* out, float a, float b) {
  float x[8];
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3f + k;
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
  float s = 0.f;
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 12345.f) out[0] = s;
}

__global__ void __launch_bounds__(256) p_dfma(double* out, double a, double b) {
  double x[8];
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < kIters / 16; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  double s = 0.0;
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 12345.0) out[0] = s;
}

__global__ void __launch_bounds__(256) p_rcp(float* out) {
  float x[8];
  for (int k = 0; k < 8; ++k) x[k] = 1.5f + threadIdx.x * 1e-3f + k;
  for (int i = 0; i < kIters / 4; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      asm volatile("rcp.approx.ftz.f32 %0, %0;" : "+f"(x[k]));
      x[k] += 1.0f;   // keeps consecutive reciprocals from folding
    }
  float s = 0.f;
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 12345.f) out[0] = s;
}

__global__ void __launch_bounds__(256) p_cvt_d2f(float* out) {
  double x[8];
  float acc[8];
  for (int k = 0; k < 8; ++k) { x[k] = 1.25 + threadIdx.x * 1e-3 + k; acc[k] = 0.f; }
  for (int i = 0; i < kIters / 16; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float f;
      asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(f) : "d"(x[k]));
      acc[k] += f;
    }
  float s = 0.f;
  for (int k = 0; k < 8; ++k) s += acc[k];
  if (s == 12345.f) out[0] = s;
}

__global__ void __launch_bounds__(256) p_ialu(unsigned* out) {
  unsigned x[8];
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 2654435761u + k;
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (x[k] ^ (x[k] >> 3)) + 0x9E3779B9u;
  unsigned s = 0;
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 12345u) out[0] = s;
}

__global__ void __launch_bounds__(256) p_copy(const float4* __restrict__ a, float4* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = a[i];
}

// splitmix64 (Steele, Lea, Flood 2014) of a counter: test bit patterns
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Integer conversions of the FP32 form against the hardware conversions.
// Pattern k: a random double (odd k: exponent confined to the FP32 range and
// its edges) and a random float bit pattern.  Inputs below the normal FP32
// range must give signed zero (the documented flush); every other input the
// hardware's result bit for bit (NaN: any NaN).
__global__ void __launch_bounds__(256) k_check_cvt(long long n, unsigned long long seed,
                                                   unsigned long long* bad) {
  unsigned long long cnt = 0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const unsigned long long r = mix64(seed ^ mix64((unsigned long long)k));
    unsigned long long db = r;
    if (k & 1) {
      const unsigned long long e = 870ull + (r >> 52) % 300ull;   // 870..1169
      db = (r & 0x800FFFFFFFFFFFFFull) | (e << 52);
    }
    if ((k & 15) == 2) db = (r & 0x8000000000000000ull) | 0x7FF0000000000000ull | ((k & 16) ? (r & 0xFFFFFull) : 0ull);
    const double x = __longlong_as_double((long long)db);
    const float hw = __double2float_rn(x), mine = crk::d2f_int(x);
    const bool below = fabs(x) < 1.1754943508222875e-38;   // 2^-126
    bool ok;
    if (x != x) ok = mine != mine;
    else if (below) ok = __float_as_uint(mine) == (unsigned)((db >> 32) & 0x80000000ull);
    else ok = __float_as_uint(mine) == __float_as_uint(hw);
    // round-toward-zero conversion of the physicality check: the hardware's
    // __double2float_rz in the normal FP32 range, signed zero below, NaN above
    const float rz = crk::d2f_rz(x);
    bool okz;
    if (((db >> 52) & 0x7FFull) >= 1151ull) okz = rz != rz;   // |x| >= 2^128, infinities, NaNs
    else if (below) okz = __float_as_uint(rz) == (unsigned)((db >> 32) & 0x80000000ull);
    else okz = __float_as_uint(rz) == __float_as_uint(__double2float_rz(x));
    const unsigned fb = (unsigned)(r >> 17);
    const float f = __uint_as_float(fb);
    const double hwd = (double)f, mined = crk::f2d_int(f);
    bool okd;
    if (f != f) okd = mined != mined;
    else if (((fb >> 23) & 0xFFu) == 0u) okd = __double_as_longlong(mined) == (long long)((unsigned long long)(fb & 0x80000000u) << 32);
    else okd = __double_as_longlong(mined) == __double_as_longlong(hwd);
    cnt += (ok ? 0u : 1u) + (okd ? 0u : 1u) + (okz ? 0u : 1u);
  }
  if (cnt) atomicAdd(bad, cnt);
}

}  // namespace

extern "C" int cr_check_conversions(long long n, unsigned long long seed, long long* mismatches) {
  if (!mismatches || n < 0) return CR_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CR_ENODEV;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CR_ECUDA;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) return CR_ENOMEM;
  unsigned long long h = 0;
  int rc = CR_OK;
  if (cudaMemset(d, 0, sizeof(h)) != cudaSuccess) rc = CR_ECUDA;
  if (rc == CR_OK && n > 0) k_check_cvt<<<sms * 8, 256>>>(n, seed, d);
  if (rc == CR_OK && (cudaGetLastError() != cudaSuccess ||
                      cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess))
    rc = CR_ECUDA;
  cudaFree(d);
  if (rc == CR_OK) *mismatches = (long long)h;
  return rc;
}

// host <-> device copy-engine bandwidth with pinned host memory (kinds 6-8)
static int probe_link(int kind, double* result) {
  const size_t bytes = (size_t)64 << 20;
  void *h_in = nullptr, *h_out = nullptr, *d_a = nullptr, *d_b = nullptr;
  cudaStream_t s1 = nullptr, s2 = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr, j2 = nullptr;
  int rc = CR_OK;
  if (cudaHostAlloc(&h_in, bytes, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&h_out, bytes, cudaHostAllocDefault) != cudaSuccess || cudaMalloc(&d_a, bytes) != cudaSuccess ||
      cudaMalloc(&d_b, bytes) != cudaSuccess)
    rc = CR_ENOMEM;
  if (rc == CR_OK && (cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess ||
                      cudaEventCreate(&j2) != cudaSuccess))
    rc = CR_ECUDA;
  float best = 1e30f;
  for (int rep = 0; rep < 5 && rc == CR_OK; ++rep) {
    cudaEventRecord(t0, s1);
    cudaStreamWaitEvent(s2, t0, 0);
    if (kind == 6 || kind == 8) cudaMemcpyAsync(d_a, h_in, bytes, cudaMemcpyHostToDevice, s1);
    if (kind == 7) cudaMemcpyAsync(h_out, d_b, bytes, cudaMemcpyDeviceToHost, s1);
    if (kind == 8) cudaMemcpyAsync(h_out, d_b, bytes, cudaMemcpyDeviceToHost, s2);
    cudaEventRecord(j2, s2);
    cudaStreamWaitEvent(s1, j2, 0);
    cudaEventRecord(t1, s1);
    if (cudaEventSynchronize(t1) != cudaSuccess) { rc = CR_ECUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (rep > 0 && ms < best) best = ms;
  }
  for (cudaEvent_t e : {t0, t1, j2})
    if (e) cudaEventDestroy(e);
  if (s1) cudaStreamDestroy(s1);
  if (s2) cudaStreamDestroy(s2);
  cudaFreeHost(h_in);
  cudaFreeHost(h_out);
  cudaFree(d_a);
  cudaFree(d_b);
  if (rc == CR_OK) *result = bytes / (best * 1e-3);
  return rc;
}

extern "C" int cr_probe_peak(int kind, double* result) {
  if (!result || kind < 0 || kind > 8) return CR_EINVAL;
  if (kind >= 6) return probe_link(kind, result);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CR_ENODEV;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CR_ECUDA;
  const int blocks = sms * 8, threads = 256;
  void* buf = nullptr;
  size_t nvec = 0;
  if (kind == 5) {
    nvec = (size_t)1 << 26;   // 2 x 1 GiB of float4
    if (cudaMalloc(&buf, 2 * nvec * sizeof(float4)) != cudaSuccess) return CR_ENOMEM;
  } else if (cudaMalloc(&buf, 64) != cudaSuccess) {
    return CR_ENOMEM;
  }
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  double ops = 0.0;
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(t0);
    switch (kind) {
      case 0: p_ffma<<<blocks, threads>>>((float*)buf, 0.999f, 1e-3f); ops = 8.0 * kIters; break;
      case 1: p_dfma<<<blocks, threads>>>((double*)buf, 0.999, 1e-3); ops = 8.0 * (kIters / 16); break;
      case 2: p_rcp<<<blocks, threads>>>((float*)buf); ops = 8.0 * (kIters / 4); break;
      case 3: p_cvt_d2f<<<blocks, threads>>>((float*)buf); ops = 8.0 * (kIters / 16); break;
      case 4: p_ialu<<<blocks, threads>>>((unsigned*)buf); ops = 8.0 * 2 * kIters; break;
      case 5: {
        const float4* a = (const float4*)buf;
        float4* b = (float4*)buf + nvec;
        p_copy<<<sms * 16, 256>>>(a, b, nvec);
        ops = 0.0;
        break;
      }
    }
    cudaEventRecord(t1);
    if (cudaEventSynchronize(t1) != cudaSuccess) { cudaFree(buf); return CR_ECUDA; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(buf);
  if (cudaGetLastError() != cudaSuccess) return CR_ECUDA;
  if (kind == 5) *result = 2.0 * nvec * sizeof(float4) / (best * 1e-3);
  else *result = ops * (double)blocks * threads / (best * 1e-3);
  return CR_OK;
}
