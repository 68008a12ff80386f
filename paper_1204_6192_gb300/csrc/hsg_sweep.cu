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
#include "hsg_device.cuh"
#include "hsg_internal.h"

namespace hsg {

template <int F, bool HB, bool J16, bool FAST, bool EN>
__global__ void __launch_bounds__(SWEEP_BS) k_half_sweep(const SweepParams p) {
  constexpr int VEC = FmtInfo<F>::VEC, PL = FmtInfo<F>::PLANES;
  using Chunk = typename FmtInfo<F>::Chunk;
  extern __shared__ float esum[];                  // [SWEEP_BS / 32][GPT * VEC] (EN only)
  const int4 blk = p.blocks[blockIdx.x];
  const SampleDev& sd = p.samples[blk.x];
  const uint32_t h = (uint32_t)blk.z + threadIdx.x;
  const uint32_t half_n = (uint32_t)sd.N >> 1;
  const bool active = h < half_n;
  if (!EN && !active) return;
  const int g0 = blk.y * p.GPT;
  const int g1 = min(p.G, g0 + p.GPT);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  SiteGeom gm;
  float j6[6], h3[3];
  uint32_t jh[6];                                  // FP16 couplings, broadcast pairs
  constexpr bool MIXED = (F == FMT_F16) && J16;
  long long nb_off[6], own_off = 0;
  const unsigned char* base = p.spins + sd.spin_off;
  const long long ps = sd.plane_stride;
  const long long gstride = (long long)sd.N * FmtInfo<F>::CHUNK;
  if (active) {
    gm = site_geom(sd, h, p.parity);
    load_record<J16>(p.rec, sd.rec_off + gm.own, j6, h3);
    if (MIXED) load_record_j16(p.rec, sd.rec_off + gm.own, jh);
#pragma unroll
    for (int n = 0; n < 6; ++n) nb_off[n] = chunk_offset<F>(sd, g0, gm.nb[n]);
    own_off = chunk_offset<F>(sd, g0, gm.own);
  }
  const uint32_t sweep = HB ? (uint32_t)(p.counters[0] + (unsigned long long)p.sweep_offset) : 0u;

  for (int g = g0; g < g1; ++g) {
    float e[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) e[v] = 0.0f;
    if (active) {
      const long long dg = (long long)(g - g0) * gstride;
      Chunk nc[6][PL];
#pragma unroll
      for (int n = 0; n < 6; ++n) load_chunks<F, true>(base + nb_off[n] + dg, ps, nc[n]);
      unsigned char* own_p = p.spins + sd.spin_off + own_off + dg;
      Chunk c[PL];
      load_chunks<F, false>(own_p, ps, c);

      // local field h = sum_n J_n s_n + H, in the order +x, -x, +y, -y, +z, -z
      Spins<VEC> hf;
      if constexpr (MIXED) {
        // FP16 spins and couplings: fused f16 x f16 + f32, bit-identical to
        // multiply-then-add because the products are exact
#pragma unroll
        for (int k = 0; k < VEC / 2; ++k) {
          hf.x[k] = make_float2(0.0f, 0.0f);
          hf.y[k] = make_float2(0.0f, 0.0f);
          hf.z[k] = make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int n = 0; n < 6; ++n) {
          fma_f16_pair(hf.x[0], nc[n][0].x, jh[n]);
          fma_f16_pair(hf.x[1], nc[n][0].y, jh[n]);
          fma_f16_pair(hf.y[0], nc[n][1].x, jh[n]);
          fma_f16_pair(hf.y[1], nc[n][1].y, jh[n]);
          fma_f16_pair(hf.z[0], nc[n][2].x, jh[n]);
          fma_f16_pair(hf.z[1], nc[n][2].y, jh[n]);
        }
      } else {
        {
          Spins<VEC> nb;
          decode<F>(nc[0], nb);
          const float2 jj = f2(j6[0]);
#pragma unroll
          for (int k = 0; k < VEC / 2; ++k) {
            hf.x[k] = mul2(jj, nb.x[k]);
            hf.y[k] = mul2(jj, nb.y[k]);
            hf.z[k] = mul2(jj, nb.z[k]);
          }
        }
#pragma unroll
        for (int n = 1; n < 6; ++n) {
          Spins<VEC> nb;
          decode<F>(nc[n], nb);
          const float2 jj = f2(j6[n]);
#pragma unroll
          for (int k = 0; k < VEC / 2; ++k) {
            hf.x[k] = add2(hf.x[k], mul2(jj, nb.x[k]));
            hf.y[k] = add2(hf.y[k], mul2(jj, nb.y[k]));
            hf.z[k] = add2(hf.z[k], mul2(jj, nb.z[k]));
          }
        }
      }
      {
        const float2 hx = f2(h3[0]), hy = f2(h3[1]), hz = f2(h3[2]);
#pragma unroll
        for (int k = 0; k < VEC / 2; ++k) {
          hf.x[k] = add2(hf.x[k], hx);
          hf.y[k] = add2(hf.y[k], hy);
          hf.z[k] = add2(hf.z[k], hz);
        }
      }

      Spins<VEC> s;
      decode<F>(c, s);
      if (HB) {
        const uint32_t sys0 = (uint32_t)sd.sys_base + (uint32_t)g * VEC;   // even
        const float* beta = p.beta + (long long)blk.x * p.Wp + g * VEC;
#pragma unroll
        for (int k = 0; k < VEC / 2; ++k) {
          const uint4 r = philox4x32_10(make_uint4(gm.site, (sys0 >> 1) + k, sweep, TAG_HB),
                                        p.seed_lo, p.seed_hi);
          hb_move<FAST>(s.x[k].x, s.y[k].x, s.z[k].x, hf.x[k].x, hf.y[k].x, hf.z[k].x,
                        beta[2 * k], u01(r.x), u01(r.y));
          hb_move<FAST>(s.x[k].y, s.y[k].y, s.z[k].y, hf.x[k].y, hf.y[k].y, hf.z[k].y,
                        beta[2 * k + 1], u01(r.z), u01(r.w));
        }
      } else {
#pragma unroll
        for (int k = 0; k < VEC / 2; ++k) or_move2(s.x[k], s.y[k], s.z[k], hf.x[k], hf.y[k], hf.z[k]);
      }
      encode<F>(s, c);
      store_chunks<F>(own_p, ps, c);

      if (EN) {
        // energy of the new state from the stored values: every bond joins one
        // odd and one even site, E = - sum_odd s_i.h_i - sum_even H_j.s_j
        Spins<VEC> st;
        decode<F>(c, st);
#pragma unroll
        for (int k = 0; k < VEC / 2; ++k) {
          float2 d;
          if (p.parity == 1) {
            d = add2(add2(mul2(st.x[k], hf.x[k]), mul2(st.y[k], hf.y[k])), mul2(st.z[k], hf.z[k]));
          } else {
            d = add2(add2(mul2(st.x[k], f2(h3[0])), mul2(st.y[k], f2(h3[1]))),
                     mul2(st.z[k], f2(h3[2])));
          }
          e[2 * k] = -d.x;
          e[2 * k + 1] = -d.y;
        }
      }
    }
    if (EN) {
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        const float t = warp_sum(e[v]);
        if (lane == 0) esum[warp * p.GPT * VEC + (g - g0) * VEC + v] = t;
      }
    }
  }
  if (EN) {
    __syncthreads();
    double* out = p.epart + ((long long)p.parity * p.n_blocks + blockIdx.x) * p.Wp;
    for (int j = threadIdx.x; j < p.Wp; j += SWEEP_BS) {
      double acc = 0.0;
      const int jj = j - g0 * VEC;
      if (jj >= 0 && jj < (g1 - g0) * VEC) {
        for (int w = 0; w < SWEEP_BS / 32; ++w) acc += (double)esum[w * p.GPT * VEC + jj];
      }
      out[j] = acc;
    }
  }
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
  }
  return cudaErrorInvalidValue;
}

}  // namespace hsg
