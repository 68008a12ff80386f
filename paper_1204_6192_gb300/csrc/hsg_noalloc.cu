// FP64 energies of caller-owned FP32 spin arrays without any device
// allocation: the block partial sums live in a fixed file-scope __device__
// array instead of memory the library would cudaMalloc.
//
// Some callers cannot let a library allocate device memory: code running
// while a CUDA graph is being captured (cudaMalloc is not allowed inside a
// capture), frameworks that hand every byte of device memory to their own
// pool allocator, and latency-critical loops where cudaMalloc/cudaFree would
// synchronise the device.  They pass their own inputs and outputs and get the
// same energies as hsg_energies, with the scratch taken from this file's
// static array.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/hsg.h"
#include "hsg_internal.h"

namespace hsg {
void set_global_error(const char* msg);
}

namespace {

// Largest scratch the entry point uses: W * ceil(N / (256 * 8)) block partials.
constexpr long long kScratchDoubles = 1ll << 19;   // 4 MiB per device
constexpr int kThreads = 256;
constexpr int kSitesPerThread = 8;
constexpr int kMaxDevices = 64;

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_energy_scratch[kScratchDoubles];

double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// One block per (chunk of sites, system w): per-site energies in FP32 with
// every bond counted once (forward bonds +x, +y, +z) plus the field term,
// summed per thread in FP64 and per block in a fixed order.
__global__ void __launch_bounds__(kThreads) k_energy_xyz(const float* __restrict__ s,
                                                         const float* __restrict__ J,
                                                         const float* __restrict__ H, int L,
                                                         int n_chunks, double* partials) {
  const int w = blockIdx.y, chunk = blockIdx.x;
  const long long N = (long long)L * L * L;
  const float* sw = s + (long long)w * N * 3;
  double acc = 0.0;
  for (int k = 0; k < kSitesPerThread; ++k) {
    const long long i = ((long long)chunk * kSitesPerThread + k) * kThreads + threadIdx.x;
    if (i >= N) break;
    const int x = (int)(i % L), y = (int)((i / L) % L), z = (int)(i / ((long long)L * L));
    const long long ix = (x + 1 == L ? i - x : i + 1);
    const long long iy = (y + 1 == L ? i - (long long)y * L : i + L);
    const long long iz = (z + 1 == L ? i - (long long)z * L * L : i + (long long)L * L);
    const float sx = sw[3 * i], sy = sw[3 * i + 1], sz = sw[3 * i + 2];
    const float jx = J[3 * i], jy = J[3 * i + 1], jz = J[3 * i + 2];
    float fx = jx * sw[3 * ix] + jy * sw[3 * iy] + jz * sw[3 * iz];
    float fy = jx * sw[3 * ix + 1] + jy * sw[3 * iy + 1] + jz * sw[3 * iz + 1];
    float fz = jx * sw[3 * ix + 2] + jy * sw[3 * iy + 2] + jz * sw[3 * iz + 2];
    if (H) {
      fx += H[3 * i];
      fy += H[3 * i + 1];
      fz += H[3 * i + 2];
    }
    acc -= (double)(sx * fx + sy * fy + sz * fz);
  }
  __shared__ double red[kThreads];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[(long long)w * n_chunks + chunk] = red[0];
}

__global__ void k_energy_xyz_final(const double* partials, int n_chunks, int W, double* E) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  double e = 0.0;
  for (int c = 0; c < n_chunks; ++c) e += partials[(long long)w * n_chunks + c];
  E[w] = e;
}

// Device address of the static scratch on the current device (looked up once
// per device, with that device current).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_energy_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" hsg_status hsg_energies_xyz_noalloc(const float* spins_dev, const float* J_dev,
                                               const float* H_dev, int L, int W, double* E_dev,
                                               void* stream) {
  if (!spins_dev || !J_dev || !E_dev) {
    hsg::set_global_error("spins, J and E must not be NULL");
    return HSG_EINVAL;
  }
  if (L < 2 || L > 512 || W < 1) {
    hsg::set_global_error("need 2 <= L <= 512 and W >= 1");
    return HSG_EINVAL;
  }
  const long long N = (long long)L * L * L;
  const long long per_chunk = (long long)kThreads * kSitesPerThread;
  const long long n_chunks = (N + per_chunk - 1) / per_chunk;
  if (W > 65535 || n_chunks * W > kScratchDoubles) {
    hsg::set_global_error("W * ceil(L^3 / 2048) exceeds the 524288 partial sums of the static scratch");
    return HSG_EINVAL;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    hsg::set_global_error(cudaGetErrorString(e));
    return HSG_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  k_energy_xyz<<<dim3((unsigned)n_chunks, (unsigned)W), kThreads, 0, st>>>(
      spins_dev, J_dev, H_dev, L, (int)n_chunks, scratch);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_energy_xyz_final<<<(W + 127) / 128, 128, 0, st>>>(scratch, (int)n_chunks, W, E_dev);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    hsg::set_global_error(cudaGetErrorString(e));
    return HSG_ECUDA;
  }
  return HSG_OK;
}
