// Reductions and bookkeeping kernels: FP64 energies (Eq. 1), the parallel
// tempering pass (Eq. 4), the overlap measurements (Eq. 5 and its
// k-dependent form), the random initial state and the conversions between
// the stored spin formats and FP32 (x, y, z).
//
// Every reduction is deterministic: per-thread partial sums, a fixed-order
// shuffle/shared-memory tree inside a block, and a second kernel that adds the
// block partials in a fixed order.  Two runs give bit-identical results.
#include "hsg_kernels.cuh"

namespace hsg {

// ---------------------------------------------------------------------------
// Energies.  Every bond joins an odd and an even site, so
//   E = - sum_{odd i} s_i . h_i  - sum_{even j} H_j . s_j
// with h_i the full local field (bonds + field) of the odd site i.
// ---------------------------------------------------------------------------
template <int F, bool J16>
__global__ void __launch_bounds__(RED_BS) k_energy(const EnergyParams p) {
  constexpr int VEC = FmtInfo<F>::VEC, PL = FmtInfo<F>::PLANES;
  using Chunk = typename FmtInfo<F>::Chunk;
  extern __shared__ float esum[];                 // [2][RED_BS / 32][GPT * VEC]
  const int4 blk = p.blocks[blockIdx.x];
  const SampleDev& sd = p.samples[blk.x];
  const uint32_t h = (uint32_t)blk.z + threadIdx.x;
  const uint32_t half_n = (uint32_t)sd.N >> 1;
  const bool active = h < half_n;
  const int g0 = blk.y * p.GPT;
  const int g1 = min(p.G, g0 + p.GPT);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int stride = p.GPT * VEC;
  float* esum_even = esum;
  float* esum_odd = esum + (RED_BS / 32) * stride;

  SiteGeom gm;                                   // the odd site with half-index h
  float j6[6], h3[3], je[6], he[3];
  long long nb_off[6], odd_off = 0, even_off = 0;
  const unsigned char* base = p.spins + sd.spin_off;
  const long long ps = sd.plane_stride;
  const long long gstride = (long long)sd.N * FmtInfo<F>::CHUNK;
  if (active) {
    gm = site_geom(sd, h, 1);
    load_record<J16>(p.rec, sd.rec_off + gm.own, j6, h3);
    load_record<J16>(p.rec, sd.rec_off + h, je, he);   // even site with the same half-index
#pragma unroll
    for (int n = 0; n < 6; ++n) nb_off[n] = chunk_offset<F>(sd, g0, gm.nb[n]);
    odd_off = chunk_offset<F>(sd, g0, gm.own);
    even_off = chunk_offset<F>(sd, g0, h);
  }
  for (int g = g0; g < g1; ++g) {
    float eo[VEC], ee[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) { eo[v] = 0.0f; ee[v] = 0.0f; }
    if (active) {
      const long long dg = (long long)(g - g0) * gstride;
      Chunk nc[6][PL], co[PL], ce[PL];
#pragma unroll
      for (int n = 0; n < 6; ++n) load_chunks<F, LD_RO>(base + nb_off[n] + dg, ps, nc[n]);
      load_chunks<F, LD_RO>(base + odd_off + dg, ps, co);
      load_chunks<F, LD_RO>(base + even_off + dg, ps, ce);
      Spins<VEC> hf, t;
      decode<F>(nc[0], t);
#pragma unroll
      for (int q = 0; q < VEC / 2; ++q) {
        hf.x[q] = mul2(f2(j6[0]), t.x[q]);
        hf.y[q] = mul2(f2(j6[0]), t.y[q]);
        hf.z[q] = mul2(f2(j6[0]), t.z[q]);
      }
#pragma unroll
      for (int n = 1; n < 6; ++n) {
        decode<F>(nc[n], t);
#pragma unroll
        for (int q = 0; q < VEC / 2; ++q) {
          hf.x[q] = fma2(f2(j6[n]), t.x[q], hf.x[q]);
          hf.y[q] = fma2(f2(j6[n]), t.y[q], hf.y[q]);
          hf.z[q] = fma2(f2(j6[n]), t.z[q], hf.z[q]);
        }
      }
      Spins<VEC> so, se;
      decode<F>(co, so);
      decode<F>(ce, se);
#pragma unroll
      for (int q = 0; q < VEC / 2; ++q) {
        const float2 hx2 = add2(hf.x[q], f2(h3[0]));
        const float2 hy2 = add2(hf.y[q], f2(h3[1]));
        const float2 hz2 = add2(hf.z[q], f2(h3[2]));
        const float2 o = dot3_2(so.x[q], so.y[q], so.z[q], hx2, hy2, hz2);
        const float2 e = dot3_2(se.x[q], se.y[q], se.z[q], f2(he[0]), f2(he[1]), f2(he[2]));
        eo[2 * q] = -o.x;
        eo[2 * q + 1] = -o.y;
        ee[2 * q] = -e.x;
        ee[2 * q + 1] = -e.y;
      }
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const float to = warp_sum(eo[v]);
      const float te = warp_sum(ee[v]);
      if (lane == 0) {
        esum_odd[warp * stride + (g - g0) * VEC + v] = to;
        esum_even[warp * stride + (g - g0) * VEC + v] = te;
      }
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < p.Wp; j += RED_BS) {
    double ae = 0.0, ao = 0.0;
    const int jj = j - g0 * VEC;
    if (jj >= 0 && jj < (g1 - g0) * VEC) {
      for (int w = 0; w < RED_BS / 32; ++w) {
        ae += (double)esum_even[w * stride + jj];
        ao += (double)esum_odd[w * stride + jj];
      }
    }
    p.partials[(long long)blockIdx.x * p.Wp + j] = ae;
    p.partials[((long long)p.n_blocks + blockIdx.x) * p.Wp + j] = ao;
  }
}

// E[s][w] = sum over the sample's blocks of the even-site and odd-site partials,
// in two fixed-order levels: split k of the sample's rows is added by a block
// of 32 systems x 8 row lanes (coalesced rows of Wp doubles), then the splits.
__global__ void __launch_bounds__(256) k_energy_final1(const EnergyParams p) {
  __shared__ double red[8][32];
  energy_final1_unit<false>(p, blockIdx.z, blockIdx.y, blockIdx.x, red);
}

// one warp per system (8 per block)
__global__ void k_energy_final2(const EnergyParams p) {
  const int gw = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (gw >= p.n_samples * p.Wp) return;
  energy_final2_warp<false>(p, gw / p.Wp, gw % p.Wp, threadIdx.x & 31);
}

cudaError_t launch_energy_final(const EnergyParams& p, cudaStream_t st) {
  k_energy_final1<<<dim3(p.splits, (p.Wp + 31) / 32, p.n_samples), 256, 0, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_energy_final2<<<(p.n_samples * p.Wp + 7) / 8, 256, 0, st>>>(p);
  return cudaGetLastError();
}

template <int F, bool J16>
static cudaError_t energy_fmt(const EnergyParams& p, cudaStream_t st) {
  const size_t smem = sizeof(float) * 2 * (RED_BS / 32) * p.GPT * FmtInfo<F>::VEC;
  k_energy<F, J16><<<p.n_blocks, RED_BS, smem, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_energy_final(p, st);
}

cudaError_t launch_energy(int fmt, bool j16, const EnergyParams& p, cudaStream_t st) {
  switch (fmt) {
    case FMT_F32: return j16 ? energy_fmt<FMT_F32, true>(p, st) : energy_fmt<FMT_F32, false>(p, st);
    case FMT_F16: return j16 ? energy_fmt<FMT_F16, true>(p, st) : energy_fmt<FMT_F16, false>(p, st);
    case FMT_BF16: return j16 ? energy_fmt<FMT_BF16, true>(p, st) : energy_fmt<FMT_BF16, false>(p, st);
    case FMT_ANG16: return j16 ? energy_fmt<FMT_ANG16, true>(p, st) : energy_fmt<FMT_ANG16, false>(p, st);
    case FMT_OCT16: return j16 ? energy_fmt<FMT_OCT16, true>(p, st) : energy_fmt<FMT_OCT16, false>(p, st);
    case FMT_YX4: return j16 ? energy_fmt<FMT_YX4, true>(p, st) : energy_fmt<FMT_YX4, false>(p, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Parallel tempering, Eq. (4): one thread per (sample, replica) chain walks the
// pairs (k, k+1) upwards from the lowest temperature; an accepted exchange
// swaps the temperatures of the two configurations.  Runs as one block so that
// the counters can be advanced after every chain is done.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_pt(const PTParams p) {
  const int n_chains = p.n_samples * p.R_O;
  for (int c = threadIdx.x; c < n_chains; c += blockDim.x) pt_chain<false>(p, c);
  __syncthreads();
  for (int s = threadIdx.x; s < p.n_samples; s += blockDim.x) {
    if (!p.active[s]) continue;
    p.counters[2 * s] += (unsigned long long)p.sweeps_per_call;
    p.counters[2 * s + 1] += (unsigned long long)p.bump_pt;
  }
}

cudaError_t launch_pt(const PTParams& p, cudaStream_t st) {
  int n = p.n_samples * p.R_O;
  int bs = n >= 1024 ? 1024 : ((n + 31) / 32) * 32;
  k_pt<<<1, bs, 0, st>>>(p);
  return cudaGetLastError();
}

// The last level of the FP64 energy sums (Eq. 1) and the PT pass (Eq. 4) in one
// block, for steps with few systems: each warp sums the level-1 partials of its
// systems (the same code and order as k_energy_final2), then, after a block
// barrier, one thread per chain walks its pairs as k_pt does.  One launch
// instead of two.  With `staged`, the permutations, energies and inverse
// temperatures are first copied into shared memory (dynamic, laid out as
// [samples][Wp] and [samples][R_T] doubles, then [chains][R_T] ints and the
// chains' uniforms [chains][R_T - 1]): each pair of a chain reads its slot's
// configuration and then that configuration's energy, two dependent loads that
// now hit shared memory instead of L2, and the uniforms are drawn by all threads
// at once instead of by each chain's thread.  The same arithmetic on the same
// values, so the same decisions.
__global__ void __launch_bounds__(1024) k_energy2_pt(const EnergyParams e, const PTParams p, int staged) {
  extern __shared__ double pt_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int gw = warp; gw < e.n_samples * e.Wp; gw += nw)
    energy_final2_warp<false>(e, gw / e.Wp, gw % e.Wp, lane);
  __syncthreads();
  const int n_chains = p.n_samples * p.R_O;
  if (staged) {
    const int np = n_chains * p.R_T, ne = p.n_samples * p.Wp, nb = p.n_samples * p.R_T;
    const int R1 = p.R_T > 1 ? p.R_T - 1 : 1, nu = n_chains * R1;
    double* sE = pt_smem;
    double* sib = sE + ne;
    int* sperm = reinterpret_cast<int*>(sib + nb);
    float* su = reinterpret_cast<float*>(sperm + np);
    for (int i = threadIdx.x; i < ne; i += blockDim.x) sE[i] = p.E[i];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sib[i] = p.inv_temps[i];
    for (int i = threadIdx.x; i < np; i += blockDim.x) sperm[i] = p.perm[i];
    if (p.bump_pt)
      for (int i = threadIdx.x; i < nu; i += blockDim.x) su[i] = pt_uniform(p, i / R1, i % R1);
    __syncthreads();
    for (int c = threadIdx.x; c < n_chains; c += blockDim.x) {
      const int s = c / p.R_O, r = c - s * p.R_O;
      pt_chain_on<false>(p, c, sperm + c * p.R_T, sE + s * p.Wp + r * p.R_T, sib + s * p.R_T,
                         su + c * R1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < np; i += blockDim.x) p.perm[i] = sperm[i];
  } else {
    for (int c = threadIdx.x; c < n_chains; c += blockDim.x) pt_chain<false>(p, c);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < p.n_samples; s += blockDim.x) {
    if (!p.active[s]) continue;
    p.counters[2 * s] += (unsigned long long)p.sweeps_per_call;
    p.counters[2 * s + 1] += (unsigned long long)p.bump_pt;
  }
}

bool energy_pt_folded(int n_samples, int Wp) { return (long long)n_samples * Wp <= ENERGY_PT_FOLD_SYSTEMS; }

cudaError_t launch_energy_final_pt(const EnergyParams& e, const PTParams& p, cudaStream_t st) {
  if (!energy_pt_folded(e.n_samples, e.Wp)) {
    cudaError_t err = launch_energy_final(e, st);
    if (err != cudaSuccess) return err;
    return launch_pt(p, st);
  }
  k_energy_final1<<<dim3(e.splits, (e.Wp + 31) / 32, e.n_samples), 256, 0, st>>>(e);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  // shared-memory copies of the chains (48 kB at most without an opt-in)
  const size_t n_chains = (size_t)p.n_samples * p.R_O;
  const size_t smem = sizeof(double) * ((size_t)p.n_samples * p.Wp + (size_t)p.n_samples * p.R_T) +
                      sizeof(int) * n_chains * p.R_T + sizeof(float) * n_chains * std::max(1, p.R_T - 1);
  const bool staged = smem <= 48 * 1024;
  k_energy2_pt<<<1, 1024, staged ? smem : 0, st>>>(e, p, staged ? 1 : 0);
  return cudaGetLastError();
}

__global__ void k_bump(unsigned long long* counters, const unsigned char* active, int n_samples,
                       int sweeps, int pts) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_samples; s += gridDim.x * blockDim.x) {
    if (!active[s]) continue;
    counters[2 * s] += (unsigned long long)sweeps;
    counters[2 * s + 1] += (unsigned long long)pts;
  }
}

cudaError_t launch_bump(unsigned long long* counters, const unsigned char* active, int n_samples,
                        int sweeps, int pts, cudaStream_t st) {
  k_bump<<<(n_samples + 255) / 256, 256, 0, st>>>(counters, active, n_samples, sweeps, pts);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Initial state and conversions.  One thread per (site, chunk), all sites.
// ---------------------------------------------------------------------------
struct ConvItem {
  const SampleDev* sd;
  uint32_t site, g, ss;
  bool ok;
};

// Block (sample, chunk g, first site): one thread per site of chunk g.
__device__ __forceinline__ ConvItem conv_item(const ConvParams& p) {
  ConvItem it;
  const int4 blk = p.blocks[blockIdx.x];
  it.sd = &p.samples[blk.x];
  it.g = (uint32_t)blk.y;
  it.site = (uint32_t)blk.z + threadIdx.x;
  const uint32_t N = (uint32_t)it.sd->N;
  it.ok = it.site < N;
  if (!it.ok) return it;
  const uint32_t L = it.sd->L;
  const uint32_t r = (__umulhi(it.site, it.sd->fdL_m) + it.site) >> it.sd->fdL_s;
  const uint32_t x = it.site - r * L;
  const uint32_t z = (__umulhi(r, it.sd->fdL_m) + r) >> it.sd->fdL_s;
  const uint32_t y = r - z * L;
  it.ss = ((x + y + z) & 1u) * (N >> 1) + (it.site >> 1);
  return it;
}

template <int F>
__global__ void k_init(const ConvParams p) {
  constexpr int VEC = FmtInfo<F>::VEC, PL = FmtInfo<F>::PLANES;
  const ConvItem it = conv_item(p);
  if (!it.ok) return;
  Spins<VEC> s;
  const uint32_t sys0 = (uint32_t)it.sd->sys_base + it.g * VEC;
#pragma unroll
  for (int k = 0; k < VEC / 2; ++k) {
    const uint4 r = philox4x32_10(make_uint4(it.site, (sys0 >> 1) + k, 0u, TAG_INIT),
                                  p.seed_lo, p.seed_hi);
    double v[2][3];
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const double u1 = (double)u01(w[2 * b]), u2 = (double)u01(w[2 * b + 1]);
      const double zc = 2.0 * u1 - 1.0;
      const double rho = 2.0 * sqrt(u1 * (1.0 - u1));
      double sp, cp;
      sincospi(2.0 * u2, &sp, &cp);
      v[b][0] = rho * cp;
      v[b][1] = rho * sp;
      v[b][2] = zc;
    }
    s.x[k] = make_float2((float)v[0][0], (float)v[1][0]);
    s.y[k] = make_float2((float)v[0][1], (float)v[1][1]);
    s.z[k] = make_float2((float)v[0][2], (float)v[1][2]);
  }
  typename FmtInfo<F>::Chunk c[PL];
  encode<F>(s, c);
  unsigned char* o = p.spins + it.sd->spin_off + chunk_offset<F>(*it.sd, it.g, it.ss);
  store_chunks<F>(o, it.sd->plane_stride, c);
}

template <int F>
__global__ void k_get(const ConvParams p) {
  constexpr int VEC = FmtInfo<F>::VEC, PL = FmtInfo<F>::PLANES;
  const ConvItem it = conv_item(p);
  if (!it.ok) return;
  const int sidx = p.blocks[blockIdx.x].x;
  const unsigned char* o = p.spins + it.sd->spin_off + chunk_offset<F>(*it.sd, it.g, it.ss);
  typename FmtInfo<F>::Chunk c[PL];
  load_chunks<F, LD_PLAIN>(o, it.sd->plane_stride, c);
  Spins<VEC> s;
  decode<F>(c, s);
  float* out = p.xyz + p.xyz_off[sidx];
  const long long N = it.sd->N;
#pragma unroll
  for (int k = 0; k < VEC / 2; ++k) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int w = (int)it.g * VEC + 2 * k + b;
      if (w < p.W) {
        float* q = out + ((long long)w * N + it.site) * 3;
        q[0] = b ? s.x[k].y : s.x[k].x;
        q[1] = b ? s.y[k].y : s.y[k].x;
        q[2] = b ? s.z[k].y : s.z[k].x;
      }
    }
  }
}

template <int F>
__global__ void k_set(const ConvParams p) {
  constexpr int VEC = FmtInfo<F>::VEC, PL = FmtInfo<F>::PLANES;
  const ConvItem it = conv_item(p);
  if (!it.ok) return;
  const int sidx = p.blocks[blockIdx.x].x;
  const float* in = p.xyz + p.xyz_off[sidx];
  const long long N = it.sd->N;
  Spins<VEC> s;
#pragma unroll
  for (int k = 0; k < VEC / 2; ++k) {
    float v[2][3];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int w = (int)it.g * VEC + 2 * k + b;
      if (w < p.W) {
        const float* q = in + ((long long)w * N + it.site) * 3;
        v[b][0] = q[0];
        v[b][1] = q[1];
        v[b][2] = q[2];
      } else {
        v[b][0] = 0.0f;
        v[b][1] = 0.0f;
        v[b][2] = 1.0f;
      }
    }
    s.x[k] = make_float2(v[0][0], v[1][0]);
    s.y[k] = make_float2(v[0][1], v[1][1]);
    s.z[k] = make_float2(v[0][2], v[1][2]);
  }
  typename FmtInfo<F>::Chunk c[PL];
  encode<F>(s, c);
  unsigned char* o = p.spins + it.sd->spin_off + chunk_offset<F>(*it.sd, it.g, it.ss);
  store_chunks<F>(o, it.sd->plane_stride, c);
}

// The heat bath's generator (round keys precomputed) on a list of counters.
__global__ void k_philox(const uint4* ctr, long long n, const SweepParams p, uint4* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10_rk(ctr[i], p.rk);
}

cudaError_t launch_philox(const uint4* ctr, long long n, const SweepParams& p, uint4* out,
                          cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_philox<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctr, n, p, out);
  return cudaGetLastError();
}

#define HSG_CONV_SWITCH(KERNEL)                                                          \
  switch (fmt) {                                                                        \
    case FMT_F32: KERNEL<FMT_F32><<<nb, 256, 0, st>>>(p); break;                        \
    case FMT_F16: KERNEL<FMT_F16><<<nb, 256, 0, st>>>(p); break;                        \
    case FMT_BF16: KERNEL<FMT_BF16><<<nb, 256, 0, st>>>(p); break;                      \
    case FMT_ANG16: KERNEL<FMT_ANG16><<<nb, 256, 0, st>>>(p); break;                    \
    case FMT_OCT16: KERNEL<FMT_OCT16><<<nb, 256, 0, st>>>(p); break;                    \
    case FMT_YX4: KERNEL<FMT_YX4><<<nb, 256, 0, st>>>(p); break;                        \
    default: return cudaErrorInvalidValue;                                              \
  }                                                                                     \
  return cudaGetLastError();

cudaError_t launch_init(int fmt, const ConvParams& p, int nb, cudaStream_t st) {
  HSG_CONV_SWITCH(k_init)
}
cudaError_t launch_get(int fmt, const ConvParams& p, int nb, cudaStream_t st) {
  HSG_CONV_SWITCH(k_get)
}
cudaError_t launch_set(int fmt, const ConvParams& p, int nb, cudaStream_t st) {
  HSG_CONV_SWITCH(k_set)
}

}  // namespace hsg
