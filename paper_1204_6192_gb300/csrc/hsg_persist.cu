// Persistent step kernel: n whole steps (n_hb heat-bath sweeps, n_or
// over-relaxation sweeps, the FP64 energy sums, one parallel-tempering pass;
// Sec. 3.2) in one cooperative launch.  Between phases every block meets at a
// grid barrier instead of a kernel boundary, which removes the launch gaps
// that dominate small, cache-resident lattices.  All blocks are co-resident
// (cooperative launch), and each barrier wait is bounded: a block that has
// waited longer than the timeout sets the error word and the kernel returns,
// which the host reports as HSG_ETIMEOUT.
#include "hsg_kernels.cuh"

namespace hsg {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bar[0]: arrivals, bar[1]: generation, bar[2]: error word.  Returns false
// when the kernel must stop (a wait ran out here or in another block).
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned long long timeout_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vb = bar;
    __threadfence();
    const unsigned int gen = vb[1];
    const unsigned int arrived = atomicAdd(&bar[0], 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (vb[1] == gen) {
        if (vb[2] != 0u) break;
        if (global_ns() - t0 > timeout_ns) {
          atomicExch(&bar[2], 1u);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ((volatile unsigned int*)bar)[2] == 0u;
}

template <int F, bool J16, bool FAST>
__global__ void __launch_bounds__(SWEEP_BS) k_persistent(const PersistParams P) {
  extern __shared__ float esum[];
  __shared__ double red[8][32];
  SweepParams sp = P.sw;
  const EnergyParams& ep = P.en;
  const int nsw = P.nhb + P.nor;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  // fault injection (host-requested): block 0 leaves at its first barrier
  // without arriving, as a lost block would; the others' waits run out
  auto sync = [&]() {
    if (P.drop_first && blockIdx.x == 0) return false;
    return grid_barrier(P.bar, P.timeout_ns);
  };
  for (int step = 0; step < P.n_steps; ++step) {
    // the sweeps of a step pass by pass: each pass is a range of the block
    // table (a group of systems) swept nsw times before the next one starts
    for (int ps = 0; ps < P.n_passes; ++ps) {
      const int b0 = P.pass_bound[ps], b1 = P.pass_bound[ps + 1];
      for (int k = 0; k < nsw; ++k) {
        const bool hb = k < P.nhb, en = (k == nsw - 1);
        sp.sweep_offset = k;
        for (int parity = 0; parity < 2; ++parity) {
          sp.parity = parity;
          for (int b = b0 + (int)blockIdx.x; b < b1; b += gridDim.x) {
            if (hb) sweep_block<F, true, J16, FAST, false, true>(sp, b, esum);
            else if (en) sweep_block<F, false, J16, false, true, true>(sp, b, esum);
            else sweep_block<F, false, J16, false, false, true>(sp, b, esum);
          }
          if (!sync()) return;
        }
      }
    }
    // energies of the final state from the partials of the last OR sweep
    const int wgs = (ep.Wp + 31) / 32;
    const int units = ep.splits * wgs * ep.n_samples;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
      const int split = u % ep.splits, rest = u / ep.splits;
      energy_final1_unit<true>(ep, rest / wgs, rest % wgs, split, red);
    }
    if (!sync()) return;
    // level 2: one warp per system (whole warps, so every lane takes part in the shuffles)
    for (int gw = tid >> 5; gw < ep.n_samples * ep.Wp; gw += nth >> 5)
      energy_final2_warp<true>(ep, gw / ep.Wp, gw % ep.Wp, threadIdx.x & 31);
    if (!sync()) return;
    for (int c = tid; c < P.pt.n_samples * P.pt.R_O; c += nth) pt_chain<true>(P.pt, c);
    if (!sync()) return;
    for (int s = tid; s < P.pt.n_samples; s += nth) {
      if (!P.pt.active[s]) continue;
      P.pt.counters[2 * s] += (unsigned long long)nsw;
      P.pt.counters[2 * s + 1] += 1ull;
    }
    if (!sync()) return;
  }
}

template <int F, bool J16, bool FAST>
static cudaError_t persist_launch(const PersistParams& P, int grid, size_t smem, cudaStream_t st) {
  void* args[] = {(void*)&P};
  return cudaLaunchCooperativeKernel((const void*)k_persistent<F, J16, FAST>, dim3(grid),
                                     dim3(SWEEP_BS), args, smem, st);
}

template <int F, bool J16, bool FAST>
static cudaError_t persist_grid(int* grid, size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent<F, J16, FAST>, SWEEP_BS, smem);
  *grid = sms * per_sm;
  return e;
}

#define HSG_PERSIST_DISPATCH(CALL)                                              \
  switch (fmt) {                                                                \
    case FMT_F32: return j16 ? (fast ? CALL(FMT_F32, true, true) : CALL(FMT_F32, true, false))       \
                             : (fast ? CALL(FMT_F32, false, true) : CALL(FMT_F32, false, false));   \
    case FMT_F16: return j16 ? (fast ? CALL(FMT_F16, true, true) : CALL(FMT_F16, true, false))       \
                             : (fast ? CALL(FMT_F16, false, true) : CALL(FMT_F16, false, false));   \
    case FMT_BF16: return j16 ? (fast ? CALL(FMT_BF16, true, true) : CALL(FMT_BF16, true, false))    \
                              : (fast ? CALL(FMT_BF16, false, true) : CALL(FMT_BF16, false, false)); \
    case FMT_ANG16: return j16 ? (fast ? CALL(FMT_ANG16, true, true) : CALL(FMT_ANG16, true, false)) \
                               : (fast ? CALL(FMT_ANG16, false, true) : CALL(FMT_ANG16, false, false)); \
    case FMT_OCT16: return j16 ? (fast ? CALL(FMT_OCT16, true, true) : CALL(FMT_OCT16, true, false)) \
                               : (fast ? CALL(FMT_OCT16, false, true) : CALL(FMT_OCT16, false, false)); \
    case FMT_YX4: return j16 ? (fast ? CALL(FMT_YX4, true, true) : CALL(FMT_YX4, true, false))       \
                             : (fast ? CALL(FMT_YX4, false, true) : CALL(FMT_YX4, false, false));   \
  }                                                                             \
  return cudaErrorInvalidValue;

cudaError_t max_persistent_grid(int fmt, bool j16, bool fast, size_t smem, int* grid) {
#define HSG_CALL_GRID(F, J, FA) persist_grid<F, J, FA>(grid, smem)
  HSG_PERSIST_DISPATCH(HSG_CALL_GRID)
#undef HSG_CALL_GRID
}

cudaError_t launch_persistent(int fmt, bool j16, bool fast, const PersistParams& P, int grid,
                              size_t smem, cudaStream_t st) {
#define HSG_CALL_LAUNCH(F, J, FA) persist_launch<F, J, FA>(P, grid, smem, st)
  HSG_PERSIST_DISPATCH(HSG_CALL_LAUNCH)
#undef HSG_CALL_LAUNCH
}

}  // namespace hsg
