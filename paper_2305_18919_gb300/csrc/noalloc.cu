// Enclosed-volume reduction for callers that must not allocate device memory.
//
// This is the volume part of the face kernel (the sum over faces of the tetrahedron volumes
// (x0 - c) . (a x b) / 6, accumulated in double with one partial per 256-face block), packaged
// as a free function whose only scratch is a fixed array in this file. It serves callers that
// cannot call cudaMalloc: a plug-in running inside a host framework that owns all device
// memory under its own pool and budget and forbids other allocations, or a latency-bound loop
// that must not pay for cudaMalloc/cudaFree, which can synchronise the whole device.
//
// The array is a file-scope __device__ variable, so every GPU that loads this library keeps
// its 32 KB until the process exits. Host code may not pass the variable's name to a kernel:
// in host code that name is a host-side stand-in, not a device address. Every call looks the
// device address up with cudaGetSymbolAddress, with the caller's device and context current,
// and passes it to the kernels. Looking it up per call (a host-side table lookup once the
// module is loaded) keeps it right when the caller runs under a context other than the
// device's primary one, or after cudaDeviceReset, where an address saved from an earlier
// call would belong to a context that no longer holds it. The first call on a device loads
// this file's device code into the current context: make it before any stream capture.
#include "iblb_internal.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int kMaxPartials = 4096;
constexpr long long kMaxFaces = (long long)kMaxPartials * kBlock;  // 1,048,576 faces

static __device__ __align__(256) double g_volume_partials[kMaxPartials];

// Device address of g_volume_partials in the current context.
cudaError_t partials_in_current_context(double **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_volume_partials);
  if (e != cudaSuccess) return e;
  *out = static_cast<double *>(p);
  return cudaSuccess;
}

// One partial volume per block of 256 faces (warp shuffles then one warp over the block's
// warps, in a fixed order). Every partial of the call is written, so nothing needs clearing.
__global__ void __launch_bounds__(kBlock) face_volume_partials_kernel(
    int nf, const double *__restrict__ q, const int *__restrict__ faces, double cx, double cy,
    double cz, double *__restrict__ partials) {
  __shared__ double warp_sum[kBlock / 32];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  double vj = 0.0;
  if (j < nf) {
    const int i0 = faces[3 * j], i1 = faces[3 * j + 1], i2 = faces[3 * j + 2];
    double x0[3], a[3], b[3];
    for (int k = 0; k < 3; k++) {
      x0[k] = q[3 * i0 + k];
      a[k] = q[3 * i1 + k] - x0[k];
      b[k] = q[3 * i2 + k] - x0[k];
    }
    const double n0 = a[1] * b[2] - a[2] * b[1];
    const double n1 = a[2] * b[0] - a[0] * b[2];
    const double n2 = a[0] * b[1] - a[1] * b[0];
    vj = ((x0[0] - cx) * n0 + (x0[1] - cy) * n1 + (x0[2] - cz) * n2) * (1.0 / 6.0);
  }
  for (int o = 16; o > 0; o >>= 1) vj += __shfl_down_sync(0xffffffffu, vj, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = vj;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? warp_sum[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
}

// Sum of the first n partials in a fixed order by one warp.
__global__ void sum_partials_kernel(const double *__restrict__ partials, int n,
                                    double *__restrict__ out) {
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += 32) v += partials[k];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) *out = v;
}

}  // namespace

extern "C" int iblb_mesh_volume_noalloc(const double *q_dev, const int32_t *faces_dev,
                                        int32_t nf, const double *centre, double *V_dev,
                                        void *cuda_stream) {
  if (!q_dev || !faces_dev || !centre || !V_dev || nf < 1) return IBLB_EINVAL;
  if ((long long)nf > kMaxFaces) return IBLB_ECAPACITY;  // before any arithmetic on nf
  const int blocks = (nf + kBlock - 1) / kBlock;
  double *partials = nullptr;
  if (partials_in_current_context(&partials) != cudaSuccess) return IBLB_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  face_volume_partials_kernel<<<blocks, kBlock, 0, s>>>(nf, q_dev, faces_dev, centre[0],
                                                        centre[1], centre[2], partials);
  if (cudaGetLastError() != cudaSuccess) return IBLB_ECUDA;
  sum_partials_kernel<<<1, 32, 0, s>>>(partials, blocks, V_dev);
  if (cudaGetLastError() != cudaSuccess) return IBLB_ECUDA;
  return IBLB_OK;
}
