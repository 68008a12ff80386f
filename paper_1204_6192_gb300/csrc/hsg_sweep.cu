// Checkerboard half-sweep kernels (Sec. 3.1): every site of one parity of
// every system of every sample is updated in parallel, with either the
// over-relaxation move (Eq. 3) or the heat-bath move (Eq. 2).  Sites of one
// parity share no bond, so the result does not depend on the order of the
// updates and a launch equals the sequential half-sweep of the oracle.
//
// One thread updates VEC systems (one 16-byte chunk per plane) of one site.
// The six neighbours belong to the other parity, which this launch only
// reads, so they go through the read-only data path; the site's coupling
// record is shared by all systems of the sample.
#include "hsg_device.cuh"
#include "hsg_internal.h"

namespace hsg {

template <int F>
__device__ __forceinline__ void load_chunks_ro(const unsigned char* p, long long plane_stride,
                                               uint4* c) {
#pragma unroll
  for (int pl = 0; pl < FmtInfo<F>::PLANES; ++pl)
    c[pl] = __ldg(reinterpret_cast<const uint4*>(p + pl * plane_stride));
}

template <int F>
__device__ __forceinline__ void load_chunks(const unsigned char* p, long long plane_stride,
                                            uint4* c) {
#pragma unroll
  for (int pl = 0; pl < FmtInfo<F>::PLANES; ++pl)
    c[pl] = *reinterpret_cast<const uint4*>(p + pl * plane_stride);
}

template <int F>
__device__ __forceinline__ void store_chunks(unsigned char* p, long long plane_stride,
                                             const uint4* c) {
#pragma unroll
  for (int pl = 0; pl < FmtInfo<F>::PLANES; ++pl)
    *reinterpret_cast<uint4*>(p + pl * plane_stride) = c[pl];
}

// Coupling/field record of one storage site: 6 bonds (+x, -x, +y, -y, +z, -z), 3 field.
template <bool J16>
__device__ __forceinline__ void load_record(const void* rec, long long idx, float* j6, float* h3) {
  if (J16) {
    const uint2* r = reinterpret_cast<const uint2*>(rec) + idx * 3;
    const uint2 a = __ldg(r), b = __ldg(r + 1), c = __ldg(r + 2);
    float2 t;
    t = h2f(a.x); j6[0] = t.x; j6[1] = t.y;
    t = h2f(a.y); j6[2] = t.x; j6[3] = t.y;
    t = h2f(b.x); j6[4] = t.x; j6[5] = t.y;
    t = h2f(b.y); h3[0] = t.x; h3[1] = t.y;
    t = h2f(c.x); h3[2] = t.x;
  } else {
    const float4* r = reinterpret_cast<const float4*>(rec) + idx * 3;
    const float4 a = __ldg(r), b = __ldg(r + 1), c = __ldg(r + 2);
    j6[0] = a.x; j6[1] = a.y; j6[2] = a.z; j6[3] = a.w;
    j6[4] = b.x; j6[5] = b.y; h3[0] = b.z; h3[1] = b.w;
    h3[2] = c.x;
  }
}

struct SiteGeom {
  uint32_t own;     // storage site of the updated spin
  uint32_t nb[6];   // storage sites of +x, -x, +y, -y, +z, -z
  uint32_t site;    // natural site index x + L (y + L z)
};

// Storage indices of a site of the given parity with half-index h and of its
// six (opposite-parity) neighbours, periodic boundaries.
__device__ __forceinline__ SiteGeom site_geom(const SampleDev& sd, uint32_t h, int parity) {
  const uint32_t L = sd.L, Lh = sd.Lh, half_n = (uint32_t)sd.N >> 1;
  const uint32_t r = (__umulhi(h, sd.fdLh_m) + h) >> sd.fdLh_s;     // row = y + L z
  const uint32_t hx = h - r * Lh;
  const uint32_t z = (__umulhi(r, sd.fdL_m) + r) >> sd.fdL_s;
  const uint32_t y = r - z * L;
  const uint32_t x = 2u * hx + ((uint32_t)(parity + y + z) & 1u);
  const uint32_t ob = (uint32_t)(1 - parity) * half_n;
  const uint32_t xp = (x + 1 == L) ? 0u : x + 1, xm = (x == 0) ? L - 1 : x - 1;
  const uint32_t yp = (y + 1 == L) ? 0u : y + 1, ym = (y == 0) ? L - 1 : y - 1;
  const uint32_t zp = (z + 1 == L) ? 0u : z + 1, zm = (z == 0) ? L - 1 : z - 1;
  const uint32_t xh = x >> 1;
  SiteGeom gm;
  gm.own = (uint32_t)parity * half_n + h;
  gm.nb[0] = ob + (xp >> 1) + r * Lh;
  gm.nb[1] = ob + (xm >> 1) + r * Lh;
  gm.nb[2] = ob + xh + (yp + L * z) * Lh;
  gm.nb[3] = ob + xh + (ym + L * z) * Lh;
  gm.nb[4] = ob + xh + (y + L * zp) * Lh;
  gm.nb[5] = ob + xh + (y + L * zm) * Lh;
  gm.site = 2u * h + (x & 1u);
  return gm;
}

template <int F, bool HB, bool J16, bool FAST, bool EN>
__global__ void __launch_bounds__(SWEEP_BS) k_half_sweep(const SweepParams p) {
  constexpr int VEC = FmtInfo<F>::VEC, PL = FmtInfo<F>::PLANES, ELEM = FmtInfo<F>::ELEM;
  const int2 blk = p.blocks[blockIdx.x];
  const SampleDev& sd = p.samples[blk.x];
  const uint32_t item = (uint32_t)blk.y + threadIdx.x;
  const uint32_t half_n = (uint32_t)sd.N >> 1;
  const bool active = item < half_n * (uint32_t)p.G;
  if (!EN && !active) return;
  float e[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) e[v] = 0.0f;

  if (active) {
    const uint32_t h = (__umulhi(item, p.fdG_m) + item) >> p.fdG_s;
    const uint32_t g = item - h * (uint32_t)p.G;
    const SiteGeom gm = site_geom(sd, h, p.parity);

    const long long site_stride = (long long)p.Wp * ELEM;
    const unsigned char* base = p.spins + sd.spin_off + (long long)g * 16;
    const long long ps = sd.plane_stride;

    float j6[6], h3[3];
    load_record<J16>(p.rec, sd.rec_off + gm.own, j6, h3);

    // local field h = sum_n J_n s_n + H, summed in the order +x, -x, +y, -y, +z, -z
    Spins<VEC> hf;
    {
      uint4 c[PL];
      Spins<VEC> nb;
      load_chunks_ro<F>(base + gm.nb[0] * site_stride, ps, c);
      decode<F>(c, nb);
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
      uint4 c[PL];
      Spins<VEC> nb;
      load_chunks_ro<F>(base + gm.nb[n] * site_stride, ps, c);
      decode<F>(c, nb);
      const float2 jj = f2(j6[n]);
#pragma unroll
      for (int k = 0; k < VEC / 2; ++k) {
        hf.x[k] = add2(hf.x[k], mul2(jj, nb.x[k]));
        hf.y[k] = add2(hf.y[k], mul2(jj, nb.y[k]));
        hf.z[k] = add2(hf.z[k], mul2(jj, nb.z[k]));
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

    unsigned char* own_p = p.spins + sd.spin_off + (long long)g * 16 + gm.own * site_stride;
    uint4 c[PL];
    Spins<VEC> s;
    load_chunks<F>(own_p, ps, c);
    decode<F>(c, s);

    if (HB) {
      const uint32_t sweep = (uint32_t)(p.counters[0] + (unsigned long long)p.sweep_offset);
      const uint32_t sys0 = (uint32_t)sd.sys_base + g * VEC;   // even
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
      // energy of the new state from the stored values: every bond joins one odd
      // and one even site, E = - sum_odd s_i.h_i - sum_even H_j.s_j
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
    __shared__ float red[SWEEP_BS][VEC];
    double* out = p.epart + ((long long)p.parity * p.n_blocks + blockIdx.x) * p.Wp;
    block_system_sums<VEC, SWEEP_BS>(e, (uint32_t)blk.y, p.G, p.Wp, out, red);
  }
}

template <int F>
static cudaError_t launch_fmt(bool hb, bool j16, bool fast, bool en, const SweepParams& p, int nb,
                              cudaStream_t st) {
  dim3 grid(nb), block(SWEEP_BS);
  if (hb) {
    if (j16) {
      if (fast) k_half_sweep<F, true, true, true, false><<<grid, block, 0, st>>>(p);
      else k_half_sweep<F, true, true, false, false><<<grid, block, 0, st>>>(p);
    } else {
      if (fast) k_half_sweep<F, true, false, true, false><<<grid, block, 0, st>>>(p);
      else k_half_sweep<F, true, false, false, false><<<grid, block, 0, st>>>(p);
    }
  } else if (en) {
    if (j16) k_half_sweep<F, false, true, false, true><<<grid, block, 0, st>>>(p);
    else k_half_sweep<F, false, false, false, true><<<grid, block, 0, st>>>(p);
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
