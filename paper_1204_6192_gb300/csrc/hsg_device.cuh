// Device-side building blocks of the sweep kernels: the Philox4x32-10
// generator, the uniform map, the spin storage codecs and the two single-spin
// moves of the method (Eq. 2 heat bath, Eq. 3 over-relaxation).
//
// Arithmetic is binary32 throughout; over-relaxation uses separately rounded
// multiplies and adds (no fused multiply-add), following the paper's warning
// that fused multiply-adds made the microcanonical moves drift (Sec. 5).
// Pairs of systems are processed together with the packed f32x2 instructions
// of sm_100+ (each lane rounds exactly like the scalar instruction).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hsg_internal.h"

namespace hsg {

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// u = (2 (x >> 9) + 1) 2^-24, exactly representable in binary32, inside (0, 1).
__device__ __forceinline__ float u01(uint32_t x) {
  return (float)(2u * (x >> 9) + 1u) * 5.9604644775390625e-8f;
}

enum { TAG_INIT = 0, TAG_HB = 1, TAG_PT = 2 };

// ----------------------------------------------------------------------------
// Packed pair arithmetic (two systems per instruction).
// ----------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}

// ----------------------------------------------------------------------------
// Storage formats.  A chunk is 16 bytes of one "plane" holding VEC systems of
// one site; component formats store 3 planes (x, y, z), packed formats 1.
// ----------------------------------------------------------------------------
template <int F> struct FmtInfo;
template <> struct FmtInfo<FMT_F32>   { static constexpr int VEC = 4, PLANES = 3, ELEM = 4; };
template <> struct FmtInfo<FMT_F16>   { static constexpr int VEC = 8, PLANES = 3, ELEM = 2; };
template <> struct FmtInfo<FMT_BF16>  { static constexpr int VEC = 8, PLANES = 3, ELEM = 2; };
template <> struct FmtInfo<FMT_ANG16> { static constexpr int VEC = 4, PLANES = 1, ELEM = 4; };
template <> struct FmtInfo<FMT_OCT16> { static constexpr int VEC = 4, PLANES = 1, ELEM = 4; };

// VEC systems of one site as FP32 pairs.
template <int VEC> struct Spins {
  float2 x[VEC / 2], y[VEC / 2], z[VEC / 2];
};

__device__ __forceinline__ float2 as_f2_lo(uint4 v) {
  return make_float2(__uint_as_float(v.x), __uint_as_float(v.y));
}
__device__ __forceinline__ float2 as_f2_hi(uint4 v) {
  return make_float2(__uint_as_float(v.z), __uint_as_float(v.w));
}
__device__ __forceinline__ float2 h2f(uint32_t w) {
  __half2 h = *reinterpret_cast<__half2*>(&w);
  return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2h(float2 v) {
  __half2 h = __floats2half2_rn(v.x, v.y);
  return *reinterpret_cast<uint32_t*>(&h);
}
// bfloat16 -> binary32 is exact: the 16 bits become the high half of the word
__device__ __forceinline__ float2 b2f(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
__device__ __forceinline__ uint32_t f2b(float2 v) {
  __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  return *reinterpret_cast<uint32_t*>(&h);
}

// --- angle pair: theta on 65536 levels of [0, pi], phi on a 2^16 ring -----
__device__ __forceinline__ void ang16_decode(uint32_t w, float& x, float& y, float& z) {
  const float tq = (float)(w & 0xffffu), pq = (float)(w >> 16);
  float st, ct, sp, cp;
  sincospif(tq * (1.0f / 65535.0f), &st, &ct);
  sincospif(pq * (1.0f / 32768.0f), &sp, &cp);
  x = st * cp;
  y = st * sp;
  z = ct;
}
__device__ __forceinline__ uint32_t ang16_encode(float x, float y, float z) {
  const float zc = fminf(1.0f, fmaxf(-1.0f, z));
  const float th = acosf(zc);
  const float ph = atan2f(y, x);
  int tq = (int)floorf(th * (65535.0f / 3.14159265358979f) + 0.5f);
  tq = min(tq, 65535);
  const int pq = ((int)floorf(ph * (65536.0f / 6.28318530717959f) + 0.5f)) & 0xffff;
  return (uint32_t)tq | ((uint32_t)pq << 16);
}

// --- octahedral map (Cigolle, Donow, Evangelakos, Mara, McGuire, Meyer,
//     JCGT 3(2), 2014) on a signed 16-bit grid --------------------------------
__device__ __forceinline__ float sgn_nn(float v) { return v >= 0.0f ? 1.0f : -1.0f; }
__device__ __forceinline__ void oct16_decode(uint32_t w, float& x, float& y, float& z) {
  const float px = (float)(int16_t)(w & 0xffffu) * (1.0f / 32767.0f);
  const float py = (float)(int16_t)(w >> 16) * (1.0f / 32767.0f);
  float vz = 1.0f - fabsf(px) - fabsf(py);
  float vx = px, vy = py;
  if (vz < 0.0f) {
    vx = (1.0f - fabsf(py)) * sgn_nn(px);
    vy = (1.0f - fabsf(px)) * sgn_nn(py);
  }
  const float inv = rsqrtf(vx * vx + vy * vy + vz * vz);
  x = vx * inv;
  y = vy * inv;
  z = vz * inv;
}
__device__ __forceinline__ uint32_t oct16_encode(float x, float y, float z) {
  const float l1 = fabsf(x) + fabsf(y) + fabsf(z);
  float px = x / l1, py = y / l1;
  if (z < 0.0f) {
    const float fx = (1.0f - fabsf(py)) * sgn_nn(px);
    const float fy = (1.0f - fabsf(px)) * sgn_nn(py);
    px = fx;
    py = fy;
  }
  px = fminf(1.0f, fmaxf(-1.0f, px));
  py = fminf(1.0f, fmaxf(-1.0f, py));
  const int qx = (int)floorf(px * 32767.0f + 0.5f);
  const int qy = (int)floorf(py * 32767.0f + 0.5f);
  return ((uint32_t)qx & 0xffffu) | (((uint32_t)qy & 0xffffu) << 16);
}

// Decode the PLANES chunks of one site into VEC FP32 spins.
template <int F>
__device__ __forceinline__ void decode(const uint4* c, Spins<FmtInfo<F>::VEC>& s) {
  if constexpr (F == FMT_F32) {
    s.x[0] = as_f2_lo(c[0]); s.x[1] = as_f2_hi(c[0]);
    s.y[0] = as_f2_lo(c[1]); s.y[1] = as_f2_hi(c[1]);
    s.z[0] = as_f2_lo(c[2]); s.z[1] = as_f2_hi(c[2]);
  } else if constexpr (F == FMT_F16 || F == FMT_BF16) {
    const uint32_t* px = reinterpret_cast<const uint32_t*>(&c[0]);
    const uint32_t* py = reinterpret_cast<const uint32_t*>(&c[1]);
    const uint32_t* pz = reinterpret_cast<const uint32_t*>(&c[2]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if constexpr (F == FMT_F16) {
        s.x[k] = h2f(px[k]); s.y[k] = h2f(py[k]); s.z[k] = h2f(pz[k]);
      } else {
        s.x[k] = b2f(px[k]); s.y[k] = b2f(py[k]); s.z[k] = b2f(pz[k]);
      }
    }
  } else {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(&c[0]);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      float x0, y0, z0, x1, y1, z1;
      if constexpr (F == FMT_ANG16) {
        ang16_decode(p[2 * k], x0, y0, z0);
        ang16_decode(p[2 * k + 1], x1, y1, z1);
      } else {
        oct16_decode(p[2 * k], x0, y0, z0);
        oct16_decode(p[2 * k + 1], x1, y1, z1);
      }
      s.x[k] = make_float2(x0, x1);
      s.y[k] = make_float2(y0, y1);
      s.z[k] = make_float2(z0, z1);
    }
  }
}

template <int F>
__device__ __forceinline__ void encode(const Spins<FmtInfo<F>::VEC>& s, uint4* c) {
  if constexpr (F == FMT_F32) {
    c[0] = make_uint4(__float_as_uint(s.x[0].x), __float_as_uint(s.x[0].y),
                      __float_as_uint(s.x[1].x), __float_as_uint(s.x[1].y));
    c[1] = make_uint4(__float_as_uint(s.y[0].x), __float_as_uint(s.y[0].y),
                      __float_as_uint(s.y[1].x), __float_as_uint(s.y[1].y));
    c[2] = make_uint4(__float_as_uint(s.z[0].x), __float_as_uint(s.z[0].y),
                      __float_as_uint(s.z[1].x), __float_as_uint(s.z[1].y));
  } else if constexpr (F == FMT_F16) {
    c[0] = make_uint4(f2h(s.x[0]), f2h(s.x[1]), f2h(s.x[2]), f2h(s.x[3]));
    c[1] = make_uint4(f2h(s.y[0]), f2h(s.y[1]), f2h(s.y[2]), f2h(s.y[3]));
    c[2] = make_uint4(f2h(s.z[0]), f2h(s.z[1]), f2h(s.z[2]), f2h(s.z[3]));
  } else if constexpr (F == FMT_BF16) {
    c[0] = make_uint4(f2b(s.x[0]), f2b(s.x[1]), f2b(s.x[2]), f2b(s.x[3]));
    c[1] = make_uint4(f2b(s.y[0]), f2b(s.y[1]), f2b(s.y[2]), f2b(s.y[3]));
    c[2] = make_uint4(f2b(s.z[0]), f2b(s.z[1]), f2b(s.z[2]), f2b(s.z[3]));
  } else {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if constexpr (F == FMT_ANG16) {
        w[2 * k] = ang16_encode(s.x[k].x, s.y[k].x, s.z[k].x);
        w[2 * k + 1] = ang16_encode(s.x[k].y, s.y[k].y, s.z[k].y);
      } else {
        w[2 * k] = oct16_encode(s.x[k].x, s.y[k].x, s.z[k].x);
        w[2 * k + 1] = oct16_encode(s.x[k].y, s.y[k].y, s.z[k].y);
      }
    }
    c[0] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Decode one system (lane w of the site's plane data) from raw storage.
template <int F>
__device__ __forceinline__ void decode_one(const unsigned char* plane0, long long plane_stride,
                                           int w, float& x, float& y, float& z) {
  if constexpr (F == FMT_F32) {
    x = reinterpret_cast<const float*>(plane0)[w];
    y = reinterpret_cast<const float*>(plane0 + plane_stride)[w];
    z = reinterpret_cast<const float*>(plane0 + 2 * plane_stride)[w];
  } else if constexpr (F == FMT_F16) {
    x = __half2float(reinterpret_cast<const __half*>(plane0)[w]);
    y = __half2float(reinterpret_cast<const __half*>(plane0 + plane_stride)[w]);
    z = __half2float(reinterpret_cast<const __half*>(plane0 + 2 * plane_stride)[w]);
  } else if constexpr (F == FMT_BF16) {
    x = __uint_as_float((uint32_t)reinterpret_cast<const uint16_t*>(plane0)[w] << 16);
    y = __uint_as_float((uint32_t)reinterpret_cast<const uint16_t*>(plane0 + plane_stride)[w] << 16);
    z = __uint_as_float((uint32_t)reinterpret_cast<const uint16_t*>(plane0 + 2 * plane_stride)[w] << 16);
  } else if constexpr (F == FMT_ANG16) {
    ang16_decode(reinterpret_cast<const uint32_t*>(plane0)[w], x, y, z);
  } else {
    oct16_decode(reinterpret_cast<const uint32_t*>(plane0)[w], x, y, z);
  }
}

// ----------------------------------------------------------------------------
// Moves
// ----------------------------------------------------------------------------

// s <- s / |s| for a pair
__device__ __forceinline__ void normalize2(float2& x, float2& y, float2& z) {
  const float2 n2 = add2(add2(mul2(x, x), mul2(y, y)), mul2(z, z));
  const float2 inv = make_float2(rsqrtf(n2.x), rsqrtf(n2.y));
  x = mul2(x, inv);
  y = mul2(y, inv);
  z = mul2(z, inv);
}

// Over-relaxation, Eq. (3), for a pair of systems: s' = 2 (s.h)/(h.h) h - s,
// unchanged where h = 0; then renormalised.
__device__ __forceinline__ void or_move2(float2& sx, float2& sy, float2& sz, float2 hx, float2 hy,
                                         float2 hz) {
  const float2 hh = add2(add2(mul2(hx, hx), mul2(hy, hy)), mul2(hz, hz));
  const float2 sh = add2(add2(mul2(sx, hx), mul2(sy, hy)), mul2(sz, hz));
  const float2 two_sh = add2(sh, sh);
  float2 f = make_float2(__fdividef(two_sh.x, hh.x), __fdividef(two_sh.y, hh.y));
  float2 nx = sub2(mul2(f, hx), sx);
  float2 ny = sub2(mul2(f, hy), sy);
  float2 nz = sub2(mul2(f, hz), sz);
  normalize2(nx, ny, nz);
  if (hh.x > 0.0f) { sx.x = nx.x; sy.x = ny.x; sz.x = nz.x; }
  if (hh.y > 0.0f) { sx.y = nx.y; sy.y = ny.y; sz.y = nz.y; }
}

// Heat bath, Eq. (2), one system: s' ~ exp(beta h.s) from the uniforms u1, u2.
// With a = beta |h| and t the angle to h, the inverse CDF of exp(a cos t) on
// [-1, 1] gives both distances to the poles in a well-conditioned form:
//   dm = 1 - cos t = -log1p((1 - u1) expm1(-2a)) / a
//   dp = 1 + cos t =  log1p(u1 expm1(2a)) / a        (dm + dp = 2)
// so sin t = sqrt(dm dp) keeps full relative accuracy near both poles (FP32
// loses it in 2 - dm when cos t is close to -1).  The azimuth is 2 pi u2 in
// the frame of Duff et al. (JCGT 6(1), 2017) around h/|h|.
template <bool FAST>
__device__ __forceinline__ void hb_move(float& sx, float& sy, float& sz, float hx, float hy,
                                        float hz, float beta, float u1, float u2) {
  const float hn = sqrtf(hx * hx + hy * hy + hz * hz);
  const float a = beta * hn;
  float dm, dp;
  if (a > 1e-12f) {
    if (FAST) {
      dm = -__logf(fmaf(1.0f - u1, __expf(-2.0f * a) - 1.0f, 1.0f)) / a;
      dp = 2.0f - dm;
    } else {
      const float inv_a = 1.0f / a;
      dm = -log1pf((1.0f - u1) * expm1f(-2.0f * a)) * inv_a;
      dp = 2.0f - dm;                   // accurate while cos t >= 0
      if (dm > 1.0f && a < 40.0f) dp = log1pf(u1 * expm1f(2.0f * a)) * inv_a;
    }
  } else {
    dm = 2.0f * (1.0f - u1);
    dp = 2.0f * u1;
  }
  dm = fminf(2.0f, fmaxf(0.0f, dm));
  dp = fminf(2.0f, fmaxf(0.0f, dp));
  const float ct = (dm <= 1.0f) ? 1.0f - dm : dp - 1.0f;
  const float st = sqrtf(dm * dp);
  float sp, cp;
  if (FAST) {
    __sincosf(6.28318530717959f * u2, &sp, &cp);
  } else {
    sincospif(2.0f * u2, &sp, &cp);
  }
  float nx = 0.0f, ny = 0.0f, nz = 1.0f;
  if (hn > 0.0f) {
    const float inv = 1.0f / hn;
    nx = hx * inv;
    ny = hy * inv;
    nz = hz * inv;
  }
  const float sg = nz >= 0.0f ? 1.0f : -1.0f;
  const float A = -1.0f / (sg + nz);
  const float B = nx * ny * A;
  const float e1x = 1.0f + sg * nx * nx * A, e1y = sg * B, e1z = -sg * nx;
  const float e2x = B, e2y = sg + ny * ny * A, e2z = -ny;
  const float px = cp * e1x + sp * e2x, py = cp * e1y + sp * e2y, pz = cp * e1z + sp * e2z;
  float ox = ct * nx + st * px, oy = ct * ny + st * py, oz = ct * nz + st * pz;
  const float inv = rsqrtf(ox * ox + oy * oy + oz * oz);
  sx = ox * inv;
  sy = oy * inv;
  sz = oz * inv;
}

// Per-block, per-system sums of the per-thread values e[VEC] of a block whose
// thread t holds item item0 + t (item = site * G + chunk g): out[g * VEC + v]
// is the sum over the threads of chunk g, added in thread order in FP64, so
// the result is independent of scheduling.  Every thread of the block calls it.
template <int VEC, int BS>
__device__ __forceinline__ void block_system_sums(const float* e, uint32_t item0, int G, int Wp,
                                                  double* out, float (*red)[VEC]) {
#pragma unroll
  for (int v = 0; v < VEC; ++v) red[threadIdx.x][v] = e[v];
  __syncthreads();
  const int r0 = (int)(item0 % (uint32_t)G);
  for (int j = threadIdx.x; j < Wp; j += BS) {
    const int g = j / VEC, v = j - (j / VEC) * VEC;
    const int t0 = (g - r0 + G) % G;
    double acc = 0.0;
    for (int t = t0; t < BS; t += G) acc += (double)red[t][v];
    out[j] = acc;
  }
  __syncthreads();
}

// Fast unsigned division by a runtime constant (Granlund & Montgomery, 1994):
// q = umulhi(n, m) + n >> s, valid for n, d < 2^31.
struct FastDiv {
  uint32_t d, m, s;
};
__device__ __forceinline__ uint32_t fdiv(uint32_t n, FastDiv f) {
  return (__umulhi(n, f.m) + n) >> f.s;
}

}  // namespace hsg
