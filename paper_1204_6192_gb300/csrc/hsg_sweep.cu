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

template <int F, bool HB, bool J16, bool FAST, bool EN, bool DEC>
__global__ void __launch_bounds__(SWEEP_BS, sweep_min_blocks<F, HB, J16, EN>()) k_half_sweep(const SweepParams p) {
  extern __shared__ float esum[];
  const int k = p.reverse ? p.n_launch - 1 - (int)blockIdx.x : (int)blockIdx.x;
  sweep_block<F, HB, J16, FAST, EN, false, DEC>(p, p.blk_base + k, esum);
}

// Decode the spins of one parity into binary32 (the chunk layout of FMT_F32,
// one parity half): each spin once, for the six neighbour loads of the next
// half-sweep.  The same decode as in the sweep, so the values are identical.
template <int F>
__global__ void __launch_bounds__(SWEEP_BS) k_decode_parity(const SweepParams p, int parity) {
  constexpr int PL = FmtInfo<F>::PLANES;
  using Chunk = typename FmtInfo<F>::Chunk;
  const int4 blk = p.blocks[p.blk_base + (int)blockIdx.x];
  if (!p.active[blk.x]) return;
  const SampleDev& sd = p.samples[blk.x];
  const uint32_t half_n = (uint32_t)sd.N >> 1;
  const uint32_t h = (uint32_t)blk.z + threadIdx.x;
  if (h >= half_n) return;
  const int g0 = blk.y * p.GPT, g1 = min(p.G, g0 + p.GPT);
  const long long gstride = (long long)sd.N * FmtInfo<F>::CHUNK;
  const unsigned char* src = p.spins + sd.spin_off + ((size_t)parity * half_n + h) * FmtInfo<F>::CHUNK;
  unsigned char* dst = const_cast<unsigned char*>(p.dec) + sd.dec_off + (size_t)h * 16;
  for (int g = g0; g < g1; ++g) {
    Chunk c[PL];
    load_chunks<F, LD_RO>(src + (long long)g * gstride, sd.plane_stride, c);
    Spins<4> s;
    decode<F>(c, s);
    uint4* d = reinterpret_cast<uint4*>(dst + (long long)g * half_n * 16);
    const long long ps = sd.dec_plane_stride / 16;
    d[0] = make_uint4(__float_as_uint(s.x[0].x), __float_as_uint(s.x[0].y), __float_as_uint(s.x[1].x),
                      __float_as_uint(s.x[1].y));
    d[ps] = make_uint4(__float_as_uint(s.y[0].x), __float_as_uint(s.y[0].y), __float_as_uint(s.y[1].x),
                       __float_as_uint(s.y[1].y));
    d[2 * ps] = make_uint4(__float_as_uint(s.z[0].x), __float_as_uint(s.z[0].y), __float_as_uint(s.z[1].x),
                           __float_as_uint(s.z[1].y));
  }
}

template <int F>
constexpr bool decodes_once() { return F == FMT_ANG16 || F == FMT_OCT16 || F == FMT_YX4; }

template <int F, bool DEC>
static cudaError_t launch_fmt_dec(bool hb, bool j16, bool fast, bool en, const SweepParams& p, int nb,
                                  cudaStream_t st) {
  dim3 grid(nb), block(SWEEP_BS);
  const size_t smem = en ? sizeof(float) * (SWEEP_BS / 32) * p.GPT * FmtInfo<F>::VEC : 0;
  if (hb) {
    if (j16) {
      if (fast) k_half_sweep<F, true, true, true, false, DEC><<<grid, block, 0, st>>>(p);
      else k_half_sweep<F, true, true, false, false, DEC><<<grid, block, 0, st>>>(p);
    } else {
      if (fast) k_half_sweep<F, true, false, true, false, DEC><<<grid, block, 0, st>>>(p);
      else k_half_sweep<F, true, false, false, false, DEC><<<grid, block, 0, st>>>(p);
    }
  } else if (en) {
    if (j16) k_half_sweep<F, false, true, false, true, DEC><<<grid, block, smem, st>>>(p);
    else k_half_sweep<F, false, false, false, true, DEC><<<grid, block, smem, st>>>(p);
  } else {
    if (j16) k_half_sweep<F, false, true, false, false, DEC><<<grid, block, 0, st>>>(p);
    else k_half_sweep<F, false, false, false, false, DEC><<<grid, block, 0, st>>>(p);
  }
  return cudaGetLastError();
}

template <int F>
static cudaError_t launch_fmt(bool hb, bool j16, bool fast, bool en, bool dec, const SweepParams& p,
                              int nb, cudaStream_t st) {
  if constexpr (decodes_once<F>()) {
    if (dec) return launch_fmt_dec<F, true>(hb, j16, fast, en, p, nb, st);
  }
  return launch_fmt_dec<F, false>(hb, j16, fast, en, p, nb, st);
}

cudaError_t launch_half_sweep(int fmt, bool hb, bool j16, bool fast, bool en, bool dec,
                              const SweepParams& p, int n_blocks, cudaStream_t st) {
  if (n_blocks <= 0) return cudaSuccess;
  switch (fmt) {
    case FMT_F32: return launch_fmt<FMT_F32>(hb, j16, fast, en, dec, p, n_blocks, st);
    case FMT_F16: return launch_fmt<FMT_F16>(hb, j16, fast, en, dec, p, n_blocks, st);
    case FMT_BF16: return launch_fmt<FMT_BF16>(hb, j16, fast, en, dec, p, n_blocks, st);
    case FMT_ANG16: return launch_fmt<FMT_ANG16>(hb, j16, fast, en, dec, p, n_blocks, st);
    case FMT_OCT16: return launch_fmt<FMT_OCT16>(hb, j16, fast, en, dec, p, n_blocks, st);
    case FMT_YX4: return launch_fmt<FMT_YX4>(hb, j16, fast, en, dec, p, n_blocks, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_decode_parity(int fmt, const SweepParams& p, int parity, int n_blocks,
                                 cudaStream_t st) {
  if (n_blocks <= 0) return cudaSuccess;
  switch (fmt) {
    case FMT_ANG16: k_decode_parity<FMT_ANG16><<<n_blocks, SWEEP_BS, 0, st>>>(p, parity); break;
    case FMT_OCT16: k_decode_parity<FMT_OCT16><<<n_blocks, SWEEP_BS, 0, st>>>(p, parity); break;
    case FMT_YX4: k_decode_parity<FMT_YX4><<<n_blocks, SWEEP_BS, 0, st>>>(p, parity); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace hsg
