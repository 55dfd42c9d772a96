// mc_selftest_math: evaluates the device arithmetic that the transport
// kernels use in place of CUDA's functions (the table-driven logarithms and
// the Newton reciprocal and square root of mc_device.cuh) side by side with
// CUDA's own log, IEEE division and IEEE square root, and the residuals of
// the hardware approximations those start from, on inputs the caller
// chooses.  A diagnostic for accuracy tests; not on the transport path.
#include <cstdint>
#include <string>

#include "../../include/mc_transport.h"
#include "mc_device.cuh"

namespace mcgpu {
void set_create_error(const std::string &msg);
}

using namespace mcgpu;

namespace {

__global__ void selftest_kernel(int fn, const unsigned long long *u, const double *x, uint64_t n, double *ours,
                                double *ref) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  switch (fn) {
    case MC_MATH_NEG_LOG_U53: {
      const unsigned long long v = u[i];
      ours[i] = neg_log_u53(v);
      ref[i] = -log(static_cast<double>(v) * 0x1.0p-53);
      break;
    }
    case MC_MATH_LOG:
      ours[i] = log_pos(x[i]);
      ref[i] = log(x[i]);
      break;
    case MC_MATH_RCP:
      ours[i] = rcp64(x[i]);
      ref[i] = 1.0 / x[i];
      break;
    case MC_MATH_SQRT:
      ours[i] = sqrt64(x[i]);
      ref[i] = sqrt(x[i]);
      break;
    default: {  // MC_MATH_APPROX
      const double v = x[i];
      double y, r;
      asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(v));
      asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(v));
      ours[i] = fma(-(v * y), y, 1.0);
      ref[i] = fma(-v, r, 1.0);
      break;
    }
  }
}

mc_status fail(const std::string &msg) {
  set_create_error("mc_selftest_math: " + msg);
  return MC_ERR_CUDA;
}

}  // namespace

extern "C" mc_status mc_selftest_math(int32_t fn, const void *in, uint64_t n, double *ours, double *ref) {
  if (fn < MC_MATH_NEG_LOG_U53 || fn > MC_MATH_APPROX) {
    set_create_error("mc_selftest_math: unknown function code");
    return MC_ERR_INVALID_ARG;
  }
  if (!in || !ours || !ref || n == 0 || n > (1ull << 28)) {
    set_create_error("mc_selftest_math: need input and output buffers and 0 < n <= 2^28");
    return MC_ERR_INVALID_ARG;
  }
  const size_t bytes = static_cast<size_t>(n) * 8;
  void *d_in = nullptr;
  double *d_ours = nullptr, *d_ref = nullptr;
  cudaError_t e = cudaMalloc(&d_in, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&d_ours, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&d_ref, bytes);
  if (e == cudaSuccess) e = cudaMemcpy(d_in, in, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
    selftest_kernel<<<blocks, 256>>>(fn, static_cast<const unsigned long long *>(d_in),
                                     static_cast<const double *>(d_in), n, d_ours, d_ref);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(ours, d_ours, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ref, d_ref, bytes, cudaMemcpyDeviceToHost);
  cudaFree(d_in);
  cudaFree(d_ours);
  cudaFree(d_ref);
  if (e != cudaSuccess) return fail(cudaGetErrorString(e));
  return MC_OK;
}
