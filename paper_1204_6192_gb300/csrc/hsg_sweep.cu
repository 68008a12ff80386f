// Checkerboard half-sweep kernels (Sec. 3.1): every site of one parity of
// every system of every sample is updated in parallel, with either the
// over-relaxation move (Eq. 3) or the heat-bath move (Eq. 2).  Sites of one
// parity share no bond, so the result does not depend on the order of the
// updates and a launch equals the sequential half-sweep of the oracle.
//
// One thread owns one site and walks a range of GPT chunks (4 systems each):
// the site geometry, the neighbour offsets and the six couplings plus field
// are computed once and reused for every chunk (the paper's reuse of J and H
// across temperatures and replicas, Sec. 3.3).  Threads of a warp hold
// consecutive sites, so every chunk load of a warp is contiguous.  The six
// neighbours belong to the other parity, which this launch only reads, so
// they go through the read-only data path.
#include "hsg_kernels.cuh"

namespace hsg {

// Both sweep kernels are latency-bound: the more warps resident per SM, the more
// loads in flight.  Bounded to 64 registers, i.e. 4 blocks (32 warps) per SM,
// every storage format but YX4 compiles with at most a few bytes of spill and
// runs 2-15 % faster than at its natural 74-104 registers (2-3 blocks per SM).
// The YX4 decode needs ~120 registers and spills heavily under any bound.
template <int F, bool HB, bool J16, bool EN>
constexpr int sweep_min_blocks() {
  return F == FMT_YX4 ? 0 : 4;
}

template <int F, bool HB, bool J16, bool FAST, bool EN>
__global__ void __launch_bounds__(SWEEP_BS, sweep_min_blocks<F, HB, J16, EN>()) k_half_sweep(const SweepParams p) {
  extern __shared__ float esum[];
  sweep_block<F, HB, J16, FAST, EN, false>(p, p.blk_base + (int)blockIdx.x, esum);
}

template <int F>
static cudaError_t launch_fmt(bool hb, bool j16, bool fast, bool en, const SweepParams& p, int nb,
                              cudaStream_t st) {
  dim3 grid(nb), block(SWEEP_BS);
  const size_t smem = en ? sizeof(float) * (SWEEP_BS / 32) * p.GPT * FmtInfo<F>::VEC : 0;
  if (hb) {
    if (j16) {
      if (fast) k_half_sweep<F, true, true, true, false><<<grid, block, 0, st>>>(p);
      else k_half_sweep<F, true, true, false, false><<<grid, block, 0, st>>>(p);
    } else {
      if (fast) k_half_sweep<F, true, false, true, false><<<grid, block, 0, st>>>(p);
      else k_half_sweep<F, true, false, false, false><<<grid, block, 0, st>>>(p);
    }
  } else if (en) {
    if (j16) k_half_sweep<F, false, true, false, true><<<grid, block, smem, st>>>(p);
    else k_half_sweep<F, false, false, false, true><<<grid, block, smem, st>>>(p);
  } else {
    if (j16) k_half_sweep<F, false, true, false, false><<<grid, block, 0, st>>>(p);
    else k_half_sweep<F, false, false, false, false><<<grid, block, 0, st>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_half_sweep(int fmt, bool hb, bool j16, bool fast, bool en,
                              const SweepParams& p, int n_blocks, cudaStream_t st) {
  if (n_blocks <= 0) return cudaSuccess;
  switch (fmt) {
    case FMT_F32: return launch_fmt<FMT_F32>(hb, j16, fast, en, p, n_blocks, st);
    case FMT_F16: return launch_fmt<FMT_F16>(hb, j16, fast, en, p, n_blocks, st);
    case FMT_BF16: return launch_fmt<FMT_BF16>(hb, j16, fast, en, p, n_blocks, st);
    case FMT_ANG16: return launch_fmt<FMT_ANG16>(hb, j16, fast, en, p, n_blocks, st);
    case FMT_OCT16: return launch_fmt<FMT_OCT16>(hb, j16, fast, en, p, n_blocks, st);
    case FMT_YX4: return launch_fmt<FMT_YX4>(hb, j16, fast, en, p, n_blocks, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hsg
