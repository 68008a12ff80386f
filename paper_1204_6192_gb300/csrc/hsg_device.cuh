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
    // one 32x32 -> 64-bit multiply per half (high and low words together)
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The same generator with the ten round keys precomputed (rk[2r], rk[2r+1] =
// key + r * Weyl constants), passed in the kernel parameters.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1], (uint32_t)p0);
  }
  return c;
}

// u = (2 (x >> 9) + 1) 2^-24, exactly representable in binary32, inside (0, 1).
// Formed from the mantissa bits: 1 + (x >> 9) 2^-23 lies in [1, 2), and
// subtracting 1 - 2^-24 leaves (2 (x >> 9) + 1) 2^-24 exactly (the operands are
// within a factor of two, so the difference is exact by Sterbenz's lemma):
// two instructions instead of an integer multiply-add, a conversion and a
// multiply.
__device__ __forceinline__ float u01(uint32_t x) {
  return __fsub_rn(__uint_as_float((x >> 9) | 0x3f800000u), __uint_as_float(0x3f7fffffu));
}

enum { TAG_INIT = 0, TAG_HB = 1, TAG_PT = 2 };

// ----------------------------------------------------------------------------
// Packed pair arithmetic (two systems per instruction).
// ----------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
// Single-instruction reciprocal and square root (at most 1 ulp from the
// correctly rounded results; the heat bath's inputs are normal numbers).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Packed binary32 pair arithmetic as PTX with an explicit rounding modifier.
// The rounding modifier does not keep the code generator from contracting a
// packed multiply whose result feeds a packed add or subtract into one fused
// multiply-add, and which pairs it contracts differs from kernel to kernel:
// an over-relaxation sweep fed with neighbours decoded by an earlier launch
// rounded its fields a few ulp away from the same sweep decoding them itself,
// and the per-half-sweep kernel's results equal a binary32 emulation in which
// every such pair is fused.  So no packed product in this code feeds a packed
// sum: each such pair is written as the fused multiply-add (fma2, dot3_2), and
// a sum that must stay unfused is formed with scalar round-to-nearest adds,
// which are never contracted.  Every kernel then rounds identically.
__device__ __forceinline__ unsigned long long f2u(float2 a) {
  return *reinterpret_cast<unsigned long long*>(&a);
}
__device__ __forceinline__ float2 u2f(unsigned long long r) {
  return *reinterpret_cast<float2*>(&r);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
  return u2f(r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
  return u2f(r);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
  return u2f(r);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)), "l"(f2u(c)));
  return u2f(r);
}
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// The dot product a.b of two pairs of 3-vectors as fma(az, bz, fma(ax, bx, ay by)).
__device__ __forceinline__ float2 dot3_2(float2 ax, float2 ay, float2 az, float2 bx, float2 by,
                                         float2 bz) {
  return fma2(az, bz, fma2(ax, bx, mul2(ay, by)));
}

// ----------------------------------------------------------------------------
// Storage formats.  A chunk holds VEC = 4 systems of one site in one "plane":
// 16 bytes (uint4) for FP32 components and for the packed 32-bit formats,
// 8 bytes (uint2) for FP16/BF16 components.  Component formats store three
// planes (x, y, z), the 16-bit pair formats one, the paper's (s_y, s_x + 4
// sign s_z) packing two (binary32 each).
// ----------------------------------------------------------------------------
template <int F> struct FmtInfo;
template <> struct FmtInfo<FMT_F32>   { static constexpr int VEC = 4, PLANES = 3, ELEM = 4, CHUNK = 16; using Chunk = uint4; };
template <> struct FmtInfo<FMT_F16>   { static constexpr int VEC = 4, PLANES = 3, ELEM = 2, CHUNK = 8;  using Chunk = uint2; };
template <> struct FmtInfo<FMT_BF16>  { static constexpr int VEC = 4, PLANES = 3, ELEM = 2, CHUNK = 8;  using Chunk = uint2; };
template <> struct FmtInfo<FMT_ANG16> { static constexpr int VEC = 4, PLANES = 1, ELEM = 4, CHUNK = 16; using Chunk = uint4; };
template <> struct FmtInfo<FMT_OCT16> { static constexpr int VEC = 4, PLANES = 1, ELEM = 4, CHUNK = 16; using Chunk = uint4; };
template <> struct FmtInfo<FMT_YX4>   { static constexpr int VEC = 4, PLANES = 2, ELEM = 4, CHUNK = 16; using Chunk = uint4; };

// VEC systems of one site as FP32 pairs.
template <int VEC> struct Spins {
  float2 x[VEC / 2], y[VEC / 2], z[VEC / 2];
};

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
__device__ __forceinline__ float2 u2f2(uint32_t a, uint32_t b) {
  return make_float2(__uint_as_float(a), __uint_as_float(b));
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
  int tq = (int)floorf(__fadd_rn(__fmul_rn(th, 65535.0f / 3.14159265358979f), 0.5f));
  tq = min(tq, 65535);
  const int pq = ((int)floorf(__fadd_rn(__fmul_rn(ph, 65536.0f / 6.28318530717959f), 0.5f))) & 0xffff;
  return (uint32_t)tq | ((uint32_t)pq << 16);
}

// --- octahedral map (Cigolle, Donow, Evangelakos, Mara, McGuire, Meyer,
//     JCGT 3(2), 2014) on a signed 16-bit grid --------------------------------
__device__ __forceinline__ float sgn_nn(float v) { return v >= 0.0f ? 1.0f : -1.0f; }
__device__ __forceinline__ void oct16_decode(uint32_t w, float& x, float& y, float& z) {
  const float px = (float)(int16_t)(w & 0xffffu) * (1.0f / 32767.0f);
  const float py = (float)(int16_t)(w >> 16) * (1.0f / 32767.0f);
  float vz = __fsub_rn(__fsub_rn(1.0f, fabsf(px)), fabsf(py));
  float vx = px, vy = py;
  if (vz < 0.0f) {
    vx = (1.0f - fabsf(py)) * sgn_nn(px);
    vy = (1.0f - fabsf(px)) * sgn_nn(py);
  }
  const float inv = rsqrtf(__fmaf_rn(vz, vz, __fmaf_rn(vy, vy, __fmul_rn(vx, vx))));
  x = __fmul_rn(vx, inv);
  y = __fmul_rn(vy, inv);
  z = __fmul_rn(vz, inv);
}
__device__ __forceinline__ uint32_t oct16_encode(float x, float y, float z) {
  const float l1 = __fadd_rn(__fadd_rn(fabsf(x), fabsf(y)), fabsf(z));
  float px = x / l1, py = y / l1;
  if (z < 0.0f) {
    const float fx = (1.0f - fabsf(py)) * sgn_nn(px);
    const float fy = (1.0f - fabsf(px)) * sgn_nn(py);
    px = fx;
    py = fy;
  }
  px = fminf(1.0f, fmaxf(-1.0f, px));
  py = fminf(1.0f, fmaxf(-1.0f, py));
  const int qx = (int)floorf(__fadd_rn(__fmul_rn(px, 32767.0f), 0.5f));
  const int qy = (int)floorf(__fadd_rn(__fmul_rn(py, 32767.0f), 0.5f));
  return ((uint32_t)qx & 0xffffu) | (((uint32_t)qy & 0xffffu) << 16);
}

// --- the paper's packing (Sec. 3.3): s_y and s_x + 4 sign(s_z), binary32 ----
// p lies in [3, 5] for s_z >= 0 and in [-5, -3] otherwise, so s_x = p - 4 sign
// is exact (Sterbenz).  s_z^2 = 1 - s_x^2 - s_y^2 is formed to about one ulp of
// its own size even near the equator: the squares as exact head + tail pairs
// (FMA), the two subtractions as error-free sums (Knuth), the error terms
// added last; then one square root.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void yx4_decode(float sy, float p, float& x, float& y, float& z) {
  const float sg = p > 2.0f ? 1.0f : -1.0f;
  const float sx = __fsub_rn(p, __fmul_rn(4.0f, sg));
  const float hx = __fmul_rn(sx, sx), lx = __fmaf_rn(sx, sx, -hx);
  const float hy = __fmul_rn(sy, sy), ly = __fmaf_rn(sy, sy, -hy);
  float s1, e1, s2, e2;
  two_sum(1.0f, -hx, s1, e1);
  two_sum(s1, -hy, s2, e2);
  const float r = __fadd_rn(s2, __fsub_rn(__fadd_rn(e1, e2), __fadd_rn(lx, ly)));
  x = sx;
  y = sy;
  z = __fmul_rn(sg, __fsqrt_rn(fmaxf(r, 0.0f)));
}
__device__ __forceinline__ void yx4_encode(float x, float y, float z, float& sy, float& p) {
  sy = y;
  p = __fadd_rn(x, z >= 0.0f ? 4.0f : -4.0f);
}

// Decode the PLANES chunks of one site into VEC = 4 FP32 spins.
template <int F>
__device__ __forceinline__ void decode(const typename FmtInfo<F>::Chunk* c, Spins<4>& s) {
  if constexpr (F == FMT_F32) {
    s.x[0] = u2f2(c[0].x, c[0].y); s.x[1] = u2f2(c[0].z, c[0].w);
    s.y[0] = u2f2(c[1].x, c[1].y); s.y[1] = u2f2(c[1].z, c[1].w);
    s.z[0] = u2f2(c[2].x, c[2].y); s.z[1] = u2f2(c[2].z, c[2].w);
  } else if constexpr (F == FMT_F16) {
    s.x[0] = h2f(c[0].x); s.x[1] = h2f(c[0].y);
    s.y[0] = h2f(c[1].x); s.y[1] = h2f(c[1].y);
    s.z[0] = h2f(c[2].x); s.z[1] = h2f(c[2].y);
  } else if constexpr (F == FMT_BF16) {
    s.x[0] = b2f(c[0].x); s.x[1] = b2f(c[0].y);
    s.y[0] = b2f(c[1].x); s.y[1] = b2f(c[1].y);
    s.z[0] = b2f(c[2].x); s.z[1] = b2f(c[2].y);
  } else if constexpr (F == FMT_YX4) {
    const uint32_t a[4] = {c[0].x, c[0].y, c[0].z, c[0].w}, b[4] = {c[1].x, c[1].y, c[1].z, c[1].w};
    float x[4], y[4], z[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) yx4_decode(__uint_as_float(a[v]), __uint_as_float(b[v]), x[v], y[v], z[v]);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      s.x[k] = make_float2(x[2 * k], x[2 * k + 1]);
      s.y[k] = make_float2(y[2 * k], y[2 * k + 1]);
      s.z[k] = make_float2(z[2 * k], z[2 * k + 1]);
    }
  } else {
    const uint32_t p[4] = {c[0].x, c[0].y, c[0].z, c[0].w};
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
__device__ __forceinline__ void encode(const Spins<4>& s, typename FmtInfo<F>::Chunk* c) {
  if constexpr (F == FMT_F32) {
    c[0] = make_uint4(__float_as_uint(s.x[0].x), __float_as_uint(s.x[0].y),
                      __float_as_uint(s.x[1].x), __float_as_uint(s.x[1].y));
    c[1] = make_uint4(__float_as_uint(s.y[0].x), __float_as_uint(s.y[0].y),
                      __float_as_uint(s.y[1].x), __float_as_uint(s.y[1].y));
    c[2] = make_uint4(__float_as_uint(s.z[0].x), __float_as_uint(s.z[0].y),
                      __float_as_uint(s.z[1].x), __float_as_uint(s.z[1].y));
  } else if constexpr (F == FMT_F16) {
    c[0] = make_uint2(f2h(s.x[0]), f2h(s.x[1]));
    c[1] = make_uint2(f2h(s.y[0]), f2h(s.y[1]));
    c[2] = make_uint2(f2h(s.z[0]), f2h(s.z[1]));
  } else if constexpr (F == FMT_BF16) {
    c[0] = make_uint2(f2b(s.x[0]), f2b(s.x[1]));
    c[1] = make_uint2(f2b(s.y[0]), f2b(s.y[1]));
    c[2] = make_uint2(f2b(s.z[0]), f2b(s.z[1]));
  } else if constexpr (F == FMT_YX4) {
    float a[4], b[4];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      yx4_encode(s.x[k].x, s.y[k].x, s.z[k].x, a[2 * k], b[2 * k]);
      yx4_encode(s.x[k].y, s.y[k].y, s.z[k].y, a[2 * k + 1], b[2 * k + 1]);
    }
    c[0] = make_uint4(__float_as_uint(a[0]), __float_as_uint(a[1]), __float_as_uint(a[2]), __float_as_uint(a[3]));
    c[1] = make_uint4(__float_as_uint(b[0]), __float_as_uint(b[1]), __float_as_uint(b[2]), __float_as_uint(b[3]));
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

// Chunk loads and stores of one site (PLANES chunks, plane_stride bytes apart).
// LD_RO: read-only path (data not written during the launch); LD_PLAIN: the
// default path; LD_CG: L2 only (data written by other blocks of a running
// persistent launch).
enum { LD_RO = 0, LD_PLAIN = 1, LD_CG = 2 };
template <int F, int POLICY>
__device__ __forceinline__ void load_chunks(const unsigned char* p, long long plane_stride,
                                            typename FmtInfo<F>::Chunk* c) {
  using C = typename FmtInfo<F>::Chunk;
#pragma unroll
  for (int pl = 0; pl < FmtInfo<F>::PLANES; ++pl) {
    const C* q = reinterpret_cast<const C*>(p + pl * plane_stride);
    c[pl] = POLICY == LD_RO ? __ldg(q) : (POLICY == LD_CG ? __ldcg(q) : *q);
  }
}

template <int F>
__device__ __forceinline__ void store_chunks(unsigned char* p, long long plane_stride,
                                             const typename FmtInfo<F>::Chunk* c) {
  using C = typename FmtInfo<F>::Chunk;
#pragma unroll
  for (int pl = 0; pl < FmtInfo<F>::PLANES; ++pl)
    *reinterpret_cast<C*>(p + pl * plane_stride) = c[pl];
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
  } else if constexpr (F == FMT_YX4) {
    yx4_decode(reinterpret_cast<const float*>(plane0)[w], reinterpret_cast<const float*>(plane0 + plane_stride)[w],
               x, y, z);
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
  const float2 n2 = dot3_2(x, y, z, x, y, z);
  const float2 inv = make_float2(rsqrtf(n2.x), rsqrtf(n2.y));
  x = mul2(x, inv);
  y = mul2(y, inv);
  z = mul2(z, inv);
}

// Over-relaxation, Eq. (3), for a pair of systems: s' = 2 (s.h)/(h.h) h - s,
// unchanged where h = 0; then renormalised.
__device__ __forceinline__ void or_move2(float2& sx, float2& sy, float2& sz, float2 hx, float2 hy,
                                         float2 hz) {
  const float2 hh = dot3_2(hx, hy, hz, hx, hy, hz);
  const float2 sh = dot3_2(sx, sy, sz, hx, hy, hz);
  const float2 two_sh = add2(sh, sh);
  float2 f = make_float2(__fdividef(two_sh.x, hh.x), __fdividef(two_sh.y, hh.y));
  float2 nx = fma2(f, hx, neg2(sx));
  float2 ny = fma2(f, hy, neg2(sy));
  float2 nz = fma2(f, hz, neg2(sz));
  normalize2(nx, ny, nz);
  if (hh.x > 0.0f) { sx.x = nx.x; sy.x = ny.x; sz.x = nz.x; }
  if (hh.y > 0.0f) { sx.y = nx.y; sy.y = ny.y; sz.y = nz.y; }
}

// (sin, cos) of 2 pi u for a uniform u in (0, 1), for one system or a pair.
// 4u is exact in binary32, so the reduction to the nearest quadrant, f = 4u - q in [-1/2, 1/2],
// is exact; r = f pi/2 lies in [-pi/4, pi/4], where the Taylor series of sin (to
// r^9) and cos (to r^10) are truncated below 3e-9; the quadrant rotation is exact.
__device__ __forceinline__ void sincos_2pi_rot(float q, float sr, float cr, float& s, float& c) {
  // rotate by q quarter turns, without branches: odd q swaps sin and cos,
  // q = 2, 3 negate sin, q = 1, 2 negate cos
  const int qi = ((int)q) & 3;
  const float a = (qi & 1) ? cr : sr;
  const float b = (qi & 1) ? sr : cr;
  s = (qi & 2) ? -a : a;
  c = ((qi + 1) & 2) ? -b : b;
}
__device__ __forceinline__ void sincos_2pi(float u, float& s, float& c) {
  const float t = __fmul_rn(4.0f, u);
  const float q = rintf(t);
  const float r = __fmul_rn(__fsub_rn(t, q), 1.57079632679489662f);
  const float r2 = __fmul_rn(r, r);
  float ps = fmaf(r2, 2.75573192e-6f, -1.98412698e-4f);
  ps = fmaf(r2, ps, 8.33333333e-3f);
  ps = fmaf(r2, ps, -1.66666667e-1f);
  const float sr = fmaf(__fmul_rn(r, r2), ps, r);
  float pc = fmaf(r2, -2.75573192e-7f, 2.48015873e-5f);
  pc = fmaf(r2, pc, -1.38888889e-3f);
  pc = fmaf(r2, pc, 4.16666667e-2f);
  pc = fmaf(r2, pc, -0.5f);
  const float cr = fmaf(r2, pc, 1.0f);
  sincos_2pi_rot(q, sr, cr, s, c);
}
__device__ __forceinline__ void sincos_2pi2(float2 u, float2& s, float2& c) {
  const float2 t = mul2(f2(4.0f), u);
  const float2 q = make_float2(rintf(t.x), rintf(t.y));
  const float2 r = mul2(sub2(t, q), f2(1.57079632679489662f));
  const float2 r2 = mul2(r, r);
  float2 ps = fma2(r2, f2(2.75573192e-6f), f2(-1.98412698e-4f));   // 1/9!, -1/7!
  ps = fma2(r2, ps, f2(8.33333333e-3f));                            // 1/5!
  ps = fma2(r2, ps, f2(-1.66666667e-1f));                           // -1/3!
  const float2 sr = fma2(mul2(r, r2), ps, r);
  float2 pc = fma2(r2, f2(-2.75573192e-7f), f2(2.48015873e-5f));   // -1/10!, 1/8!
  pc = fma2(r2, pc, f2(-1.38888889e-3f));                           // -1/6!
  pc = fma2(r2, pc, f2(4.16666667e-2f));                            // 1/4!
  pc = fma2(r2, pc, f2(-0.5f));                                     // -1/2!
  const float2 cr = fma2(r2, pc, f2(1.0f));
  sincos_2pi_rot(q.x, sr.x, cr.x, s.x, c.x);
  sincos_2pi_rot(q.y, sr.y, cr.y, s.y, c.y);
}

// Heat bath, Eq. (2): s' ~ exp(beta h.s) from the uniforms u1, u2.  With
// a = beta |h| and t the angle to h, the inverse CDF of exp(a cos t) on [-1, 1]
// gives both distances to the poles in a well-conditioned form:
//   dm = 1 - cos t = -log1p((1 - u1) expm1(-2a)) / a
//   dp = 1 + cos t =  log1p(u1 expm1(2a)) / a        (dm + dp = 2)
// so sin t = sqrt(dm dp) keeps full relative accuracy near both poles (FP32
// loses it in 2 - dm when cos t is close to -1).  The azimuth is 2 pi u2 in
// the frame of Duff et al. (JCGT 6(1), 2017) around h/|h|.
//
// hb_poles is the scalar part (one system: branches on a and on the side of
// the equator); hb_move2 moves two systems with packed pair arithmetic around
// it.  Every product and sum is an explicit round-to-nearest operation, so no
// kernel that inlines these functions can round them differently.
template <bool FAST>
__device__ __forceinline__ void hb_poles(float a, float u1, float& dm, float& dp) {
  if (a > 1e-12f) {
    const float inv_a = rcp_approx(a);
    const float om = __fsub_rn(1.0f, u1);
    // 1 - cos t = -log(y) / a with y = 1 + (1 - u1) expm1(-2a) = u1 + (1 - u1) e^{-2a}.
    // For a >= 0.35 y is formed as that sum of two positive terms (one fused
    // multiply-add, no cancellation): the form 1 + (1 - u1) (e^{-2a} - 1) loses
    // the e^{-2a} term once e^{-2a} is below half an ulp of 1 (a > ~8.7), which
    // moved cos t by up to ~e^{-a} / a for draws near the equator (u1 ~ e^{-a}).
    // Below a = 0.35, y is close to 1 and log1p of (1 - u1) expm1(-2a) keeps
    // its accuracy (for a < ~3e-8, e^{-2a} - 1 would be exactly 0 and the spin
    // would snap onto h).
    if (FAST) {
      dm = (a >= 0.35f) ? __fmul_rn(-__logf(__fmaf_rn(om, __expf(-2.0f * a), u1)), inv_a)
                        : __fmul_rn(-__logf(__fmaf_rn(om, expm1f(-2.0f * a), 1.0f)), inv_a);
      dp = __fsub_rn(2.0f, dm);
    } else {
      // the hardware exp's relative error (<~ 2a * 6e-8) enters 1 - cos t as
      // <~ 1.2e-7 absolute
      dm = (a >= 0.35f) ? __fmul_rn(-logf(__fmaf_rn(om, __expf(-2.0f * a), u1)), inv_a)
                        : __fmul_rn(-log1pf(__fmul_rn(om, expm1f(-2.0f * a))), inv_a);
      dp = __fsub_rn(2.0f, dm);                     // accurate while cos t >= 0
      if (dm > 1.0f && a < 40.0f) {
        // southern hemisphere: dp from its own form, and dm = 2 - dp (in [1, 2],
        // so accurate); the direct dm cancels there when u1 is small, since
        // 1 + (1 - u1) expm1(-2a) is then close to u1 (a = 7.7, u1 = 1.6e-5:
        // ~1e-3 relative in dm, which reached the spin through sin t)
        const float ep = (a >= 0.35f) ? __fsub_rn(__expf(2.0f * a), 1.0f) : expm1f(2.0f * a);
        dp = __fmul_rn(log1pf(__fmul_rn(u1, ep)), inv_a);
        dm = __fsub_rn(2.0f, dp);
      }
    }
  } else {
    dm = __fmul_rn(2.0f, __fsub_rn(1.0f, u1));
    dp = __fmul_rn(2.0f, u1);
  }
  dm = fminf(2.0f, fmaxf(0.0f, dm));
  dp = fminf(2.0f, fmaxf(0.0f, dp));
}

template <bool FAST>
__device__ __forceinline__ void hb_move2(float2& sx, float2& sy, float2& sz, float2 hx, float2 hy,
                                         float2 hz, float2 beta, float2 u1, float2 u2) {
  const float2 hn2 = fma2(hz, hz, fma2(hy, hy, mul2(hx, hx)));
  const bool zx = !(hn2.x > 0.0f), zy = !(hn2.y > 0.0f);
  const float2 rs = make_float2(zx ? 0.0f : rsqrtf(hn2.x), zy ? 0.0f : rsqrtf(hn2.y));   // 1/|h|
  const float2 a = mul2(beta, mul2(hn2, rs));                                             // beta |h|
  float2 dm, dp;
  hb_poles<FAST>(a.x, u1.x, dm.x, dp.x);
  hb_poles<FAST>(a.y, u1.y, dm.y, dp.y);
  const float2 ct = make_float2((dm.x <= 1.0f) ? __fsub_rn(1.0f, dm.x) : __fsub_rn(dp.x, 1.0f),
                                (dm.y <= 1.0f) ? __fsub_rn(1.0f, dm.y) : __fsub_rn(dp.y, 1.0f));
  const float2 dd = mul2(dm, dp);
  const float2 st = make_float2(sqrt_approx(dd.x), sqrt_approx(dd.y));
  float2 sp, cp;
  if (FAST) {
    const float2 w = mul2(f2(6.28318530717959f), sub2(u2, f2(0.5f)));
    __sincosf(w.x, &sp.x, &cp.x);
    __sincosf(w.y, &sp.y, &cp.y);
    sp = make_float2(-sp.x, -sp.y);
    cp = make_float2(-cp.x, -cp.y);
  } else {
    sincos_2pi2(u2, sp, cp);
  }
  float2 nx = mul2(hx, rs), ny = mul2(hy, rs), nz = mul2(hz, rs);
  if (zx) { nx.x = 0.0f; ny.x = 0.0f; nz.x = 1.0f; }
  if (zy) { nx.y = 0.0f; ny.y = 0.0f; nz.y = 1.0f; }
  const float2 sg = make_float2(nz.x >= 0.0f ? 1.0f : -1.0f, nz.y >= 0.0f ? 1.0f : -1.0f);
  const float2 sn = make_float2(__fadd_rn(sg.x, nz.x), __fadd_rn(sg.y, nz.y));   // unfused, as in hb_move
  const float2 A = make_float2(-rcp_approx(sn.x), -rcp_approx(sn.y));
  const float2 B = mul2(mul2(nx, ny), A);
  const float2 e1x = fma2(sg, mul2(mul2(nx, nx), A), f2(1.0f));
  const float2 e1y = mul2(sg, B);
  const float2 sgnx = mul2(sg, nx);
  const float2 e1z = make_float2(-sgnx.x, -sgnx.y);
  const float2 e2x = B, e2y = fma2(mul2(ny, ny), A, sg), e2z = make_float2(-ny.x, -ny.y);
  const float2 px = fma2(sp, e2x, mul2(cp, e1x));
  const float2 py = fma2(sp, e2y, mul2(cp, e1y));
  const float2 pz = fma2(sp, e2z, mul2(cp, e1z));
  const float2 ox = fma2(st, px, mul2(ct, nx));
  const float2 oy = fma2(st, py, mul2(ct, ny));
  const float2 oz = fma2(st, pz, mul2(ct, nz));
  const float2 n2 = fma2(oz, oz, fma2(oy, oy, mul2(ox, ox)));
  const float2 inv = make_float2(rsqrtf(n2.x), rsqrtf(n2.y));
  sx = mul2(ox, inv);
  sy = mul2(oy, inv);
  sz = mul2(oz, inv);
}

// The same move for one system, in the same operations and order (so the two
// give identical bits).  The tile kernel uses it: with two systems in flight
// the packed form needs more registers than its occupancy leaves.
template <bool FAST>
__device__ __forceinline__ void hb_move(float& sx, float& sy, float& sz, float hx, float hy,
                                        float hz, float beta, float u1, float u2) {
  const float hn2 = __fmaf_rn(hz, hz, __fmaf_rn(hy, hy, __fmul_rn(hx, hx)));
  const bool zero = !(hn2 > 0.0f);
  const float rs = zero ? 0.0f : rsqrtf(hn2);
  const float a = __fmul_rn(beta, __fmul_rn(hn2, rs));
  float dm, dp;
  hb_poles<FAST>(a, u1, dm, dp);
  const float ct = (dm <= 1.0f) ? __fsub_rn(1.0f, dm) : __fsub_rn(dp, 1.0f);
  const float st = sqrt_approx(__fmul_rn(dm, dp));
  float sp, cp;
  if (FAST) {
    __sincosf(__fmul_rn(6.28318530717959f, __fsub_rn(u2, 0.5f)), &sp, &cp);
    sp = -sp;
    cp = -cp;
  } else {
    sincos_2pi(u2, sp, cp);
  }
  float nx = 0.0f, ny = 0.0f, nz = 1.0f;
  if (!zero) {
    nx = __fmul_rn(hx, rs);
    ny = __fmul_rn(hy, rs);
    nz = __fmul_rn(hz, rs);
  }
  const float sg = nz >= 0.0f ? 1.0f : -1.0f;
  const float A = -rcp_approx(__fadd_rn(sg, nz));
  const float B = __fmul_rn(__fmul_rn(nx, ny), A);
  const float e1x = __fmaf_rn(sg, __fmul_rn(__fmul_rn(nx, nx), A), 1.0f);
  const float e1y = __fmul_rn(sg, B), e1z = -__fmul_rn(sg, nx);
  const float e2x = B, e2y = __fmaf_rn(__fmul_rn(ny, ny), A, sg), e2z = -ny;
  const float px = __fmaf_rn(sp, e2x, __fmul_rn(cp, e1x));
  const float py = __fmaf_rn(sp, e2y, __fmul_rn(cp, e1y));
  const float pz = __fmaf_rn(sp, e2z, __fmul_rn(cp, e1z));
  const float ox = __fmaf_rn(st, px, __fmul_rn(ct, nx));
  const float oy = __fmaf_rn(st, py, __fmul_rn(ct, ny));
  const float oz = __fmaf_rn(st, pz, __fmul_rn(ct, nz));
  const float inv = rsqrtf(__fmaf_rn(oz, oz, __fmaf_rn(oy, oy, __fmul_rn(ox, ox))));
  sx = __fmul_rn(ox, inv);
  sy = __fmul_rn(oy, inv);
  sz = __fmul_rn(oz, inv);
}

// ----------------------------------------------------------------------------
// Lattice geometry and couplings
// ----------------------------------------------------------------------------
struct SiteGeom {
  uint32_t own;     // storage site of the updated spin
  uint32_t nb[6];   // storage sites of +x, -x, +y, -y, +z, -z
  uint32_t site;    // natural site index x + L (y + L z)
};

// Storage indices of the site of the given parity with half-index h and of its
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

// The six couplings of a site as binary16 bit patterns, each broadcast to both
// halves of a 32-bit word (FP16 records only).
__device__ __forceinline__ void load_record_j16(const void* rec, long long idx, uint32_t* j2) {
  const uint2* r = reinterpret_cast<const uint2*>(rec) + idx * 3;
  const uint2 a = __ldg(r), b = __ldg(r + 1);
  const uint32_t w[3] = {a.x, a.y, b.x};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    j2[2 * k] = (w[k] & 0xffffu) * 0x10001u;
    j2[2 * k + 1] = (w[k] >> 16) * 0x10001u;
  }
}

// a += s * j for two systems, s and j binary16 (packed), a binary32.  The
// product of two binary16 numbers is exact in binary32, so this mixed-precision
// fused multiply-add rounds exactly like a multiply followed by an add.
__device__ __forceinline__ void fma_f16_pair(float2& a, uint32_t s2, uint32_t j2) {
  asm("{\n\t.reg .f16 s0, s1, j0, j1;\n\t"
      "mov.b32 {s0, s1}, %2;\n\t"
      "mov.b32 {j0, j1}, %3;\n\t"
      "fma.rn.f32.f16 %0, s0, j0, %0;\n\t"
      "fma.rn.f32.f16 %1, s1, j1, %1;\n\t}"
      : "+f"(a.x), "+f"(a.y)
      : "r"(s2), "r"(j2));
}

// Byte offset of chunk g of storage site ss in plane 0 of a sample's block.
template <int F>
__device__ __forceinline__ long long chunk_offset(const SampleDev& sd, uint32_t g, uint32_t ss) {
  return ((long long)g * sd.N + ss) * FmtInfo<F>::CHUNK;
}

// Sum of v over the 32 lanes of a warp, result in lane 0 (fixed order).
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// The warp sums of four values per lane, scattered over the lanes: lanes 0-7
// end with the sum of a[0], 8-15 of a[1], 16-23 of a[2], 24-31 of a[3].  Each
// sum pairs the lanes exactly as warp_sum does (l with l + 16, then + 8, + 4,
// + 2, + 1) and a + b equals b + a in IEEE arithmetic, so every sum equals
// warp_sum's bit for bit, with 6 shuffles and 6 additions instead of 20 each.
__device__ __forceinline__ float warp_sum4_scatter(const float* a, int lane) {
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
  const float k0 = h16 ? a[2] : a[0], k1 = h16 ? a[3] : a[1];
  const float o0 = h16 ? a[0] : a[2], o1 = h16 ? a[1] : a[3];
  const float s0 = k0 + __shfl_xor_sync(0xffffffffu, o0, 16);
  const float s1 = k1 + __shfl_xor_sync(0xffffffffu, o1, 16);
  float v = (h8 ? s1 : s0) + __shfl_xor_sync(0xffffffffu, h8 ? s0 : s1, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
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
