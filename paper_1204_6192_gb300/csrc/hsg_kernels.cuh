// Device bodies shared by the per-phase kernels and the persistent step
// kernel: one block's share of a half-sweep (Sec. 3.1, Eqs. 2-3), one unit of
// the FP64 energy reduction (Eq. 1) and one parallel-tempering chain (Eq. 4).
#pragma once

#include "hsg_device.cuh"
#include "hsg_internal.h"

namespace hsg {

// One block's share of a half-sweep: virtual block `bidx` of the sweep block
// table.  CG: every load of data written during the launch bypasses L1 (for
// the persistent kernel, whose blocks see each other's writes across grid
// barriers).  DEC: the neighbours come decoded from p.dec (packed formats).
// esum: shared memory [SWEEP_BS / 32][GPT * VEC] (EN only).
template <int F, bool HB, bool J16, bool FAST, bool EN, bool CG, bool DEC = false>
__device__ __forceinline__ void sweep_block(const SweepParams& p, int bidx, float* esum) {
  constexpr int VEC = FmtInfo<F>::VEC, PL = FmtInfo<F>::PLANES;
  using Chunk = typename FmtInfo<F>::Chunk;
  const int4 blk = p.blocks[bidx];
  if (!p.active[blk.x]) return;   // a frozen sample (the whole block belongs to it)
  const SampleDev& sd = p.samples[blk.x];
  const uint32_t h = (uint32_t)blk.z + threadIdx.x;
  const uint32_t half_n = (uint32_t)sd.N >> 1;
  bool active = h < half_n;
  if (!EN && !active) return;
  const int g0 = blk.y * p.GPT;
  const int g1 = min(p.G, g0 + p.GPT);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  SiteGeom gm;
  float j6[6], h3[3];
  uint32_t jh[6];                                  // FP16 couplings, broadcast pairs
  constexpr bool MIXED = (F == FMT_F16) && J16;
  const unsigned char* base = p.spins + sd.spin_off;
  const long long ps = sd.plane_stride;
  const long long gstride = (long long)sd.N * FmtInfo<F>::CHUNK;
  // Chunk addresses: group g of every plane starts at base + g * gstride, and a
  // site's chunk lies ss * CHUNK bytes further.  The plain sweeps keep the 32-bit
  // site indices and form each address per chunk group (fewer live registers:
  // OR half-sweep 0.179 -> 0.174 ms at L = 128, FP16); the sweeps that also sum
  // energies keep 64-bit offsets from group g0, which spill less there.
  long long nb_off[6], own_off = 0;
  if (active) {
    gm = site_geom(sd, h, p.parity);
    {
      // HSG_CHECK builds: the site in this parity's half, its neighbours in the
      // other half, the chunk groups within the sample (else skip the site)
      const uint32_t own0 = (uint32_t)p.parity * half_n, nb0 = (uint32_t)(1 - p.parity) * half_n;
      bool bad = HSG_OUT_OF_BOUNDS(gm.own >= own0 && gm.own < own0 + half_n && g1 <= p.G, p.bounds_err);
#pragma unroll
      for (int n = 0; n < 6; ++n)
        bad = bad || HSG_OUT_OF_BOUNDS(gm.nb[n] >= nb0 && gm.nb[n] < nb0 + half_n, p.bounds_err);
      if (bad) {
        active = false;
        if (!EN) return;
      }
    }
  }
  if (active) {
    load_record<J16>(p.rec, sd.rec_off + gm.own, j6, h3);
    if (MIXED) load_record_j16(p.rec, sd.rec_off + gm.own, jh);
    if constexpr (EN) {
#pragma unroll
      for (int n = 0; n < 6; ++n) nb_off[n] = chunk_offset<F>(sd, g0, gm.nb[n]);
      own_off = chunk_offset<F>(sd, g0, gm.own);
    }
  }
  const uint32_t sweep =
      HB ? (uint32_t)((CG ? __ldcg(p.counters + 2 * blk.x) : p.counters[2 * blk.x]) +
                      (unsigned long long)p.sweep_offset)
         : 0u;

  // DEC: the decoded opposite parity, chunk (g, h') at dec + (g N/2 + h') 16 bytes
  const unsigned char* decb = DEC ? p.dec + sd.dec_off : nullptr;
  const uint32_t ob = (uint32_t)(1 - p.parity) * half_n;

  for (int g = g0; g < g1; ++g) {
    float e[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) e[v] = 0.0f;
    if (active) {
      Chunk nc[DEC ? 1 : 6][PL];
      uint4 ncd[DEC ? 6 : 1][3];
      unsigned char* own_p;
      if constexpr (DEC) {
        const unsigned char* dg = decb + (long long)g * half_n * 16;
#pragma unroll
        for (int n = 0; n < 6; ++n)
          load_chunks<FMT_F32, CG ? LD_CG : LD_RO>(dg + (size_t)(gm.nb[n] - ob) * 16, sd.dec_plane_stride, ncd[n]);
        own_p = p.spins + sd.spin_off + (long long)g * gstride + (size_t)gm.own * FmtInfo<F>::CHUNK;
      } else if constexpr (EN) {
        const long long dg = (long long)(g - g0) * gstride;
#pragma unroll
        for (int n = 0; n < 6; ++n) load_chunks<F, CG ? LD_CG : LD_RO>(base + nb_off[n] + dg, ps, nc[n]);
        // (the address of the own chunk after the neighbour loads: fewer live registers)
        own_p = p.spins + sd.spin_off + own_off + dg;
      } else {
        const unsigned char* base_g = base + (long long)g * gstride;
#pragma unroll
        for (int n = 0; n < 6; ++n)
          load_chunks<F, CG ? LD_CG : LD_RO>(base_g + (size_t)gm.nb[n] * FmtInfo<F>::CHUNK, ps, nc[n]);
        own_p = p.spins + sd.spin_off + (long long)g * gstride + (size_t)gm.own * FmtInfo<F>::CHUNK;
      }
      Chunk c[PL];
      load_chunks<F, CG ? LD_CG : LD_PLAIN>(own_p, ps, c);

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
          if constexpr (DEC) decode<FMT_F32>(ncd[0], nb);
          else decode<F>(nc[0], nb);
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
          if constexpr (DEC) decode<FMT_F32>(ncd[n], nb);
          else decode<F>(nc[n], nb);
          const float2 jj = f2(j6[n]);
#pragma unroll
          for (int k = 0; k < VEC / 2; ++k) {
            hf.x[k] = fma2(jj, nb.x[k], hf.x[k]);
            hf.y[k] = fma2(jj, nb.y[k], hf.y[k]);
            hf.z[k] = fma2(jj, nb.z[k], hf.z[k]);
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
        float bt[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) bt[v] = CG ? __ldcg(beta + v) : beta[v];
#pragma unroll
        for (int k = 0; k < VEC / 2; ++k) {
          const uint4 r = philox4x32_10_rk(make_uint4(gm.site, (sys0 >> 1) + k, sweep, TAG_HB),
                                           p.rk);
          hb_move2<FAST>(s.x[k], s.y[k], s.z[k], hf.x[k], hf.y[k], hf.z[k],
                         make_float2(bt[2 * k], bt[2 * k + 1]), make_float2(u01(r.x), u01(r.z)),
                         make_float2(u01(r.y), u01(r.w)));
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
            d = dot3_2(st.x[k], st.y[k], st.z[k], hf.x[k], hf.y[k], hf.z[k]);
          } else {
            d = dot3_2(st.x[k], st.y[k], st.z[k], f2(h3[0]), f2(h3[1]), f2(h3[2]));
          }
          e[2 * k] = -d.x;
          e[2 * k + 1] = -d.y;
        }
      }
    }
    if (EN) {
      static_assert(VEC == 4, "the scattered warp sum takes four systems per chunk");
      const float t = warp_sum4_scatter(e, lane);
      if ((lane & 7) == 0) esum[warp * p.GPT * VEC + (g - g0) * VEC + (lane >> 3)] = t;
    }
  }
  if (EN) {
    __syncthreads();
    double* out = p.epart + ((long long)p.parity * p.n_blocks + bidx) * p.Wp;
    for (int j = threadIdx.x; j < p.Wp; j += SWEEP_BS) {
      double acc = 0.0;
      const int jj = j - g0 * VEC;
      if (jj >= 0 && jj < (g1 - g0) * VEC) {
        for (int w = 0; w < SWEEP_BS / 32; ++w) acc += (double)esum[w * p.GPT * VEC + jj];
      }
      out[j] = acc;
    }
    __syncthreads();   // esum is reused by the next virtual block of this block
  }
}

// ---------------------------------------------------------------------------
// FP64 energy sums.  Level 1: split `split` of the sample's block rows, systems
// 32*wg .. 32*wg+31, on 256 threads = 32 systems x 8 row lanes.  Level 2: the
// splits of one system.  Fixed order throughout.
// ---------------------------------------------------------------------------
template <bool CG>
__device__ __forceinline__ void energy_final1_unit(const EnergyParams& p, int s, int wg, int split,
                                                   double (*red)[32]) {
  if (!p.active[s]) return;   // frozen sample: its energies stand (block-uniform)
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int w = wg * 32 + tx;
  const SampleDev& sd = p.samples[s];
  const int nrows = sd.blk1 - sd.blk0;
  const int per = (nrows + p.splits - 1) / p.splits;
  const int r0 = sd.blk0 + split * per;
  const int r1 = min(r0 + per, sd.blk1);
  double acc = 0.0;
  if (w < p.Wp) {
    for (int r = r0 + ty; r < r1; r += 8) {
      const double* a = p.partials + (long long)r * p.Wp + w;
      const double* b = p.partials + ((long long)p.n_blocks + r) * p.Wp + w;
      acc += CG ? __ldcg(a) : *a;
      acc += CG ? __ldcg(b) : *b;
    }
  }
  red[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && w < p.Wp) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k][tx];
    p.partials2[((long long)s * p.splits + split) * p.Wp + w] = t;
  }
  __syncthreads();
}

// Level 2 for system w of sample s, one warp: lane j adds splits j, j + 32, ...
// in order, then the lanes are added by a fixed shuffle tree.
template <bool CG>
__device__ __forceinline__ void energy_final2_warp(const EnergyParams& p, int s, int w, int lane) {
  if (!p.active[s]) return;
  double e = 0.0;
  for (int k = lane; k < p.splits; k += 32) {
    const double* a = p.partials2 + ((long long)s * p.splits + k) * p.Wp + w;
    e += CG ? __ldcg(a) : *a;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
  if (lane == 0) p.E[(long long)s * p.Wp + w] = e;
}

// Metropolis decision of a PT pair (Eq. 4): accept iff x >= 0 or u < exp(x),
// decided exactly as in binary64.  u >= 2^-24 > exp(-17), so x < -17 always
// rejects.  Otherwise exp is evaluated in FP32 (expf: within 2 ulp; rounding
// x to FP32 adds at most 17 * 2^-24 relative), and only a u within 4e-6
// relative of it goes to the FP64 exp.  (GB300's FP64 rate is a small fraction
// of its FP32 rate and this chain is sequential.)
__device__ __forceinline__ bool pt_accept(double x, float u) {
  if (x >= 0.0) return true;
  if (x < -17.0) return false;
  const float e = expf((float)x);
  if (u < e * (1.0f - 4e-6f)) return true;
  if (u > e * (1.0f + 4e-6f)) return false;
  return (double)u < exp(x);
}

// Parallel tempering, Eq. (4), for chain c = (sample, replica): pairs (k, k+1)
// from the lowest temperature up, accepted with min[1, exp(dbeta dE)]; an
// accepted exchange swaps the temperatures of the two configurations; then
// the chain's systems get their new inverse temperatures.  Diagnostics of the
// temperature random walk (Sec. 4): per slot, the passes after which the
// configuration that held it has moved (p_diff = moved / passes), and per
// configuration the closed loops T_1 -> T_R -> T_1 (tunnelling events).
// The chain's permutation row, energies and inverse temperatures are read (and
// the permutation written) through perm, E and ib: the global arrays, or copies
// in shared memory (then CG is false and the caller writes perm back).  uf: the
// chain's R_T - 1 uniforms, drawn beforehand (same counters), or null.
template <bool CG>
__device__ __forceinline__ void pt_chain_on(const PTParams& p, int c, int* perm, const double* E,
                                            const double* ib, const float* uf = nullptr) {
  const int s = c / p.R_O, r = c - s * p.R_O;
  if (!p.active[s]) return;
  // the sample's own PT pass counter keys its random numbers
  const uint32_t step = (uint32_t)(CG ? __ldcg(p.counters + 2 * s + 1) : p.counters[2 * s + 1]);
  if (p.bump_pt) {
    unsigned long long* moved = p.moved + (long long)c * p.R_T;
    bool prev_acc = false;
    // the uniforms do not depend on the decisions: they are drawn 32 pairs at a
    // time ahead of the sequential chain, so the Philox evaluations overlap
    float uk[32];
    for (int k = 0; k + 1 < p.R_T; ++k) {
      if (!uf && (k & 31) == 0) {
#pragma unroll 4
        for (int j = 0; j < 32; ++j)
          uk[j] = (k + j + 1 < p.R_T)
                      ? u01(philox4x32_10(make_uint4((uint32_t)(k + j), (uint32_t)c, step, TAG_PT),
                                          p.seed_lo, p.seed_hi).x)
                      : 1.0f;
      }
      const int a = perm[k], b = perm[k + 1];
      const double dbeta = ib[k + 1] - ib[k];
      const double dE = (CG ? __ldcg(E + b) : E[b]) - (CG ? __ldcg(E + a) : E[a]);
      const double x = dbeta * dE;
      const bool acc = pt_accept(x, uf ? uf[k] : uk[k & 31]);
      // the configuration that held slot k before the pass moved iff pair (k-1, k)
      // moved it down or, failing that, pair (k, k+1) moved it up
      if (acc || prev_acc) moved[k] += 1ull;
      prev_acc = acc;
      if (acc) {
        perm[k] = b;
        perm[k + 1] = a;
        p.accepted[(long long)c * (p.R_T - 1) + k] += 1ull;
      }
    }
    if (p.R_T > 1) {
      if (prev_acc) moved[p.R_T - 1] += 1ull;
      // tunnelling: a configuration that reaches T_1 after T_R after T_1 closes a loop
      unsigned char* ts = p.tstate + (long long)c * p.R_T;
      unsigned int* tn = p.tunnel + (long long)c * p.R_T;
      const int bottom = perm[0], top = perm[p.R_T - 1];
      if (ts[bottom] == 2) tn[bottom] += 1u;
      ts[bottom] = 1;
      if (ts[top] == 1) ts[top] = 2;
    }
  }
  float* beta = p.beta + (long long)s * p.Wp + r * p.R_T;
  for (int t = 0; t < p.R_T; ++t) beta[perm[t]] = (float)ib[t];
}

// The uniform of pair k of chain c in the current PT pass (as pt_chain_on draws it).
__device__ __forceinline__ float pt_uniform(const PTParams& p, int c, int k) {
  const int s = c / p.R_O;
  const uint32_t step = (uint32_t)p.counters[2 * s + 1];
  return u01(philox4x32_10(make_uint4((uint32_t)k, (uint32_t)c, step, TAG_PT), p.seed_lo, p.seed_hi).x);
}

template <bool CG>
__device__ __forceinline__ void pt_chain(const PTParams& p, int c) {
  const int s = c / p.R_O, r = c - s * p.R_O;
  pt_chain_on<CG>(p, c, p.perm + (long long)c * p.R_T, p.E + (long long)s * p.Wp + r * p.R_T,
                  p.inv_temps + (long long)s * p.R_T);
}

}  // namespace hsg
