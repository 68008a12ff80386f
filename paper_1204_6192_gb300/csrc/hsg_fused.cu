// Fused over-relaxation sweep: both half-sweeps of the double checkerboard
// (Sec. 3.1, Eq. 3) in one launch, every spin read once and written once.
//
// A block walks a column of the lattice -- one chunk group (4 systems) of one
// sample, a band of ny rows of y (all x), a range of planes [za, zb) -- as a
// wavefront along z.  At plane t it updates the even sites of plane t (from the
// odd sites of planes t-1, t, t+1, all still old), then the odd sites of plane
// t-1 (from the even sites of planes t-2, t-1, t, all already new).  That is
// the order of the two half-sweeps: every even site sees only old odd spins and
// every odd site only new even spins, so the result equals the even half-sweep
// followed by the odd one, bit for bit (the same arithmetic in the same order
// as the per-half-sweep kernel).
//
// The sweep reads one spin buffer and writes the other, so blocks never wait
// for one another: the even sites a band's odd rows need from its neighbours
// (rows y0-1 and y0+ny) and those a segment needs from the planes beyond it
// (za-1 and zb) are recomputed from the old spins.  Odd and even spins reach
// shared memory by bulk copies (cp.async.bulk) into two rings of plane slots
// (odd: 6, even: 4), each with a full mbarrier.  Thread 0 issues the copies:
// the first ones at the start, then, after every step, into the slots that
// step released (the consumers are past a block barrier there), running ahead
// into the block's next work item.  The six bonds and the field of a site
// (shared by all chunk groups, so mostly L2 hits) are loaded one plane ahead.
// Every wait is bounded: one that runs out sets the error word and the block
// winds down after its copies have landed.
#include <type_traits>

#include "hsg_async.cuh"
#include "hsg_device.cuh"
#include "hsg_internal.h"

namespace hsg {

namespace {

constexpr int FD1 = 6;          // odd-site plane slots
constexpr int FD0 = 4;          // even-site plane slots
constexpr int FCW = FUSED_CONSUMER_WARPS;
constexpr int FNCT = FCW * 32;  // consumer threads
constexpr int FMAXI = 2;        // sites per consumer thread and half-step (host-checked)

__device__ __forceinline__ void consumer_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(FNCT) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Geometry of one work item (one column of one chunk group).
struct FItem {
  int s, g, y0, ny, za, zb;
  int L, Lh, hp0, hp1, R0, R1;   // halo rows of the even / odd slots, rows per slot
  bool full;                     // the band is the whole plane (rows wrap in the slot)
};

__device__ __forceinline__ FItem item_geom(const FusedParams& p, int it) {
  const int4 v = p.items[it];
  FItem f;
  f.s = v.x;
  f.g = v.y;
  f.y0 = v.z & 0xffff;
  f.ny = v.z >> 16;
  f.za = (int)(short)(v.w & 0xffff);
  f.zb = v.w >> 16;
  const SampleDev& sd = p.samples[f.s];
  f.L = sd.L;
  f.Lh = sd.Lh;
  f.full = f.ny == f.L;
  f.hp0 = f.full ? 0 : 1;
  f.hp1 = f.full ? 0 : 2;
  f.R0 = f.ny + 2 * f.hp0;
  f.R1 = f.ny + 2 * f.hp1;
  return f;
}

__device__ __forceinline__ int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// ---------------------------------------------------------------------------
// producer: bulk copies of rows [ya, ya + R) (mod L) of one parity of plane q
// ---------------------------------------------------------------------------
template <int F>
__device__ __forceinline__ void copy_plane(const FusedParams& p, const FItem& f, const SampleDev& sd,
                                           int parity, int q, int ya, int R, unsigned char* slot,
                                           uint64_t* bar) {
  constexpr int CH = FmtInfo<F>::CHUNK, PL = FmtInfo<F>::PLANES;
  const uint32_t RB = (uint32_t)f.Lh * CH;
  const uint32_t bytes = (uint32_t)PL * R * RB;
  mbar_expect_tx(bar, bytes);
  const int L = f.L;
  q = ((q % L) + L) % L;
  ya = ((ya % L) + L) % L;
  const int n1 = min(R, L - ya);
  const long long gstride = (long long)sd.N * CH;
  const long long base_ss = (long long)parity * (sd.N >> 1) + (long long)f.Lh * L * q;
#pragma unroll
  for (int c = 0; c < PL; ++c) {
    const unsigned char* g0 = p.src + sd.spin_off + c * sd.plane_stride + f.g * gstride;
    unsigned char* d = slot + (uint32_t)c * R * RB;
    bulk_copy_g2s(d, g0 + (base_ss + (long long)f.Lh * ya) * CH, (uint32_t)n1 * RB, bar);
    if (n1 < R) bulk_copy_g2s(d + (uint32_t)n1 * RB, g0 + base_ss * CH, (uint32_t)(R - n1) * RB, bar);
  }
}

// ---------------------------------------------------------------------------
// consumer: one site update from chunks in shared memory
// ---------------------------------------------------------------------------
template <bool J16>
struct Rec {
  // FP16 records: the 12 halves as three 8-byte words; FP32: three float4
  typename std::conditional<J16, uint2, float4>::type w[3];
};

template <bool J16>
__device__ __forceinline__ void load_rec(const void* rec, long long idx, Rec<J16>& r) {
  if constexpr (J16) {
    const uint2* q = reinterpret_cast<const uint2*>(rec) + idx * 3;
    r.w[0] = __ldg(q);
    r.w[1] = __ldg(q + 1);
    r.w[2] = __ldg(q + 2);
  } else {
    const float4* q = reinterpret_cast<const float4*>(rec) + idx * 3;
    r.w[0] = __ldg(q);
    r.w[1] = __ldg(q + 1);
    r.w[2] = __ldg(q + 2);
  }
}

// Couplings and field of this thread's sites of step j (even sites of plane
// t = za - 1 + j, odd sites of plane t - 1).
template <bool J16>
__device__ __forceinline__ void load_step_recs(const void* rec, const FItem& f, long long rbase,
                                               long long half, int j, const int* r0a, const int* xa,
                                               const int* rba, const int* xba, Rec<J16>* r0,
                                               Rec<J16>* r1) {
  const int L = f.L, Lh = f.Lh;
  const int t = f.za - 1 + j;
  const int zq = wrap(t, L), zq1 = wrap(t - 1, L);
#pragma unroll
  for (int k = 0; k < FMAXI; ++k) {
    if (r0a[k] >= 0) {
      const int y = wrap(f.y0 - f.hp0 + r0a[k], L);
      load_rec<J16>(rec, rbase + (long long)Lh * (y + (long long)L * zq) + xa[k], r0[k]);
    }
    if (rba[k] >= 0 && j >= 2) {
      const int y = f.y0 + rba[k];
      load_rec<J16>(rec, rbase + half + (long long)Lh * (y + (long long)L * zq1) + xba[k], r1[k]);
    }
  }
}

template <int F>
__device__ __forceinline__ void lds_chunks(const unsigned char* p, uint32_t plane_bytes,
                                           typename FmtInfo<F>::Chunk* c) {
  using C = typename FmtInfo<F>::Chunk;
#pragma unroll
  for (int pl = 0; pl < FmtInfo<F>::PLANES; ++pl) c[pl] = *reinterpret_cast<const C*>(p + pl * plane_bytes);
}
template <int F>
__device__ __forceinline__ void sts_chunks(unsigned char* p, uint32_t plane_bytes,
                                           const typename FmtInfo<F>::Chunk* c) {
  using C = typename FmtInfo<F>::Chunk;
#pragma unroll
  for (int pl = 0; pl < FmtInfo<F>::PLANES; ++pl) *reinterpret_cast<C*>(p + pl * plane_bytes) = c[pl];
}

// The over-relaxation move of one site's chunk (4 systems), with the field
// summed in the order +x, -x, +y, -y, +z, -z, then + H: the operations of the
// per-half-sweep kernel, so both give identical bits.
template <int F, bool J16>
__device__ __forceinline__ void or_chunk(const typename FmtInfo<F>::Chunk (*nc)[FmtInfo<F>::PLANES],
                                         typename FmtInfo<F>::Chunk* c, const Rec<J16>& r) {
  constexpr int VEC = FmtInfo<F>::VEC;
  constexpr bool MIXED = (F == FMT_F16) && J16;
  float j6[6], h3[3];
  if constexpr (J16) {
    float2 t;
    t = h2f(r.w[0].x); j6[0] = t.x; j6[1] = t.y;
    t = h2f(r.w[0].y); j6[2] = t.x; j6[3] = t.y;
    t = h2f(r.w[1].x); j6[4] = t.x; j6[5] = t.y;
    t = h2f(r.w[1].y); h3[0] = t.x; h3[1] = t.y;
    t = h2f(r.w[2].x); h3[2] = t.x;
  } else {
    j6[0] = r.w[0].x; j6[1] = r.w[0].y; j6[2] = r.w[0].z; j6[3] = r.w[0].w;
    j6[4] = r.w[1].x; j6[5] = r.w[1].y; h3[0] = r.w[1].z; h3[1] = r.w[1].w;
    h3[2] = r.w[2].x;
  }
  Spins<VEC> hf;
  if constexpr (MIXED) {
    uint32_t jh[6];
    const uint32_t w[3] = {r.w[0].x, r.w[0].y, r.w[1].x};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      jh[2 * k] = (w[k] & 0xffffu) * 0x10001u;
      jh[2 * k + 1] = (w[k] >> 16) * 0x10001u;
    }
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
#pragma unroll
  for (int k = 0; k < VEC / 2; ++k) or_move2(s.x[k], s.y[k], s.z[k], hf.x[k], hf.y[k], hf.z[k]);
  encode<F>(s, c);
}

}  // namespace

// Thread 0's queue of bulk copies: the odd-plane loads of every item of the
// block (planes za-2 .. zb+1) and its even-plane loads (za-1 .. zb), each issued
// as soon as a slot of its ring has been released, running into the next item.
struct CopyCursor {
  int it;         // current item (n_items: done)
  int m;          // next load within the item
  uint32_t k;     // loads issued
};

template <int F>
__device__ __forceinline__ void advance(const FusedParams& p, CopyCursor& c, int parity, uint32_t limit,
                                        unsigned char* ring, uint32_t slot_bytes, uint64_t* full,
                                        uint32_t D) {
  while (c.k < limit && c.it < p.n_items) {
    const FItem f = item_geom(p, c.it);
    const int n = f.zb - f.za + (parity ? 4 : 2);
    if (!p.active[f.s] || c.m >= n) {
      c.it += gridDim.x;
      c.m = 0;
      continue;
    }
    const SampleDev& sd = p.samples[f.s];
    const int q = parity ? f.za - 2 + c.m : f.za - 1 + c.m;
    copy_plane<F>(p, f, sd, parity, q, f.y0 - (parity ? f.hp1 : f.hp0), parity ? f.R1 : f.R0,
                  ring + (size_t)(c.k % D) * slot_bytes, full + c.k % D);
    ++c.m;
    ++c.k;
  }
}

template <int F, bool J16>
__global__ void __launch_bounds__(FNCT, 1) k_fused_or(const FusedParams p) {
  constexpr int CH = FmtInfo<F>::CHUNK, PL = FmtInfo<F>::PLANES;
  using Chunk = typename FmtInfo<F>::Chunk;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full1 = reinterpret_cast<uint64_t*>(smem);
  uint64_t* full0 = full1 + FD1;
  volatile int* s_abort = reinterpret_cast<volatile int*>(full0 + FD0);
  unsigned char* ring1 = smem + FUSED_SMEM_HEAD;
  unsigned char* ring0 = ring1 + (size_t)FD1 * p.slot1;
  const int ct = threadIdx.x;
  CopyCursor c1{(int)blockIdx.x, 0, 0u}, c0{(int)blockIdx.x, 0, 0u};   // thread 0 only
  if (ct == 0) {
    for (int k = 0; k < FD1; ++k) mbar_init(full1 + k, 1);
    for (int k = 0; k < FD0; ++k) mbar_init(full0 + k, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    advance<F>(p, c1, 1, FD1, ring1, p.slot1, full1, FD1);
    advance<F>(p, c0, 0, FD0, ring0, p.slot0, full0, FD0);
  }
  __syncthreads();

  uint32_t k1 = 0, k0 = 0;   // loads consumed (and released) before the current item
  bool aborted = false;
  for (int it = blockIdx.x; it < p.n_items && !aborted; it += gridDim.x) {
    const FItem f = item_geom(p, it);
    if (!p.active[f.s]) continue;
    const SampleDev& sd = p.samples[f.s];
    const int L = f.L, Lh = f.Lh;
    const int nsteps = f.zb - f.za + 2;
    const uint32_t RB = (uint32_t)Lh * CH;
    const uint32_t pb1 = (uint32_t)f.R1 * RB, pb0 = (uint32_t)f.R0 * RB;
    const int nP0 = f.R0 * Lh, nP1 = f.ny * Lh;
    const long long gstride = (long long)sd.N * CH;
    const long long ps = sd.plane_stride;
    unsigned char* dstg = p.dst + sd.spin_off + f.g * gstride;
    const long long half = sd.N >> 1;
    const long long rbase = sd.rec_off;
    // this thread's sites: slot row and half-x of its even sites, band row and half-x of its odd sites
    int r0a[FMAXI], xa[FMAXI], rba[FMAXI], xba[FMAXI];
#pragma unroll
    for (int k = 0; k < FMAXI; ++k) {
      const int i = ct + k * FNCT;
      const int q0 = (int)((__umulhi((uint32_t)i, sd.fdLh_m) + (uint32_t)i) >> sd.fdLh_s);
      r0a[k] = i < nP0 ? q0 : -1;
      xa[k] = i - q0 * Lh;
      rba[k] = i < nP1 ? q0 : -1;
      xba[k] = i - q0 * Lh;
    }
    Rec<J16> rc0[FMAXI], rc1[FMAXI], rn0[FMAXI], rn1[FMAXI];
    load_step_recs<J16>(p.rec, f, rbase, half, 0, r0a, xa, rba, xba, rn0, rn1);
    for (int j = 0; j < nsteps; ++j) {
      const int t = f.za - 1 + j;
#pragma unroll
      for (int k = 0; k < FMAXI; ++k) {
        rc0[k] = rn0[k];
        rc1[k] = rn1[k];
      }
      if (j + 1 < nsteps) load_step_recs<J16>(p.rec, f, rbase, half, j + 1, r0a, xa, rba, xba, rn0, rn1);
      bool ok = true;
      if (j == 0) {
        for (uint32_t m = 0; m < 3; ++m)
          ok = ok && mbar_wait(full1 + (k1 + m) % FD1, ((k1 + m) / FD1) & 1u, p.timeout_ns);
      } else {
        const uint32_t k = k1 + j + 2;
        ok = mbar_wait(full1 + k % FD1, (k / FD1) & 1u, p.timeout_ns);
      }
      {
        const uint32_t k = k0 + j;
        ok = ok && mbar_wait(full0 + k % FD0, (k / FD0) & 1u, p.timeout_ns);
      }
      if (!ok) {
        atomicOr(p.err, 1u);
        *s_abort = 1;
      }
      if (!*s_abort) {
        // even sites of plane t from the old odd sites of planes t-1, t, t+1
        const unsigned char* s1m = ring1 + (size_t)((k1 + j) % FD1) * p.slot1;
        const unsigned char* s1c = ring1 + (size_t)((k1 + j + 1) % FD1) * p.slot1;
        const unsigned char* s1p = ring1 + (size_t)((k1 + j + 2) % FD1) * p.slot1;
        unsigned char* s0c = ring0 + (size_t)((k0 + j) % FD0) * p.slot0;
        const bool write0 = t >= f.za && t < f.zb;
        const int zq = wrap(t, L);
#pragma unroll
        for (int k = 0; k < FMAXI; ++k) {
          if (r0a[k] < 0) continue;
          const int r0 = r0a[k], xh = xa[k];
          const int o = (f.y0 - f.hp0 + r0 + t) & 1;
          const int r1 = r0 + (f.hp1 - f.hp0);
          int xp = xh + o, xm = xh + o - 1;
          if (xp == Lh) xp = 0;
          if (xm < 0) xm = Lh - 1;
          int ryp = r1 + 1, rym = r1 - 1;
          if (f.full) {
            if (ryp == L) ryp = 0;
            if (rym < 0) rym = L - 1;
          }
          Chunk nc[6][PL];
          lds_chunks<F>(s1c + r1 * RB + xp * CH, pb1, nc[0]);
          lds_chunks<F>(s1c + r1 * RB + xm * CH, pb1, nc[1]);
          lds_chunks<F>(s1c + ryp * RB + xh * CH, pb1, nc[2]);
          lds_chunks<F>(s1c + rym * RB + xh * CH, pb1, nc[3]);
          lds_chunks<F>(s1p + r1 * RB + xh * CH, pb1, nc[4]);
          lds_chunks<F>(s1m + r1 * RB + xh * CH, pb1, nc[5]);
          unsigned char* own = s0c + r0 * RB + xh * CH;
          Chunk c[PL];
          lds_chunks<F>(own, pb0, c);
          or_chunk<F, J16>(nc, c, rc0[k]);
          sts_chunks<F>(own, pb0, c);
          if (write0 && r0 >= f.hp0 && r0 < f.hp0 + f.ny) {
            const int y = f.y0 + r0 - f.hp0;
            const long long ss = (long long)Lh * (y + (long long)L * zq) + xh;
#pragma unroll
            for (int pl = 0; pl < PL; ++pl) *reinterpret_cast<Chunk*>(dstg + pl * ps + ss * CH) = c[pl];
          }
        }
        // the even slot is refilled by bulk copies (async proxy) once released
        fence_proxy_async_smem();
      }
      consumer_bar();
      if (!*s_abort && j >= 2) {
        // odd sites of plane t-1 from the new even sites of planes t-2, t-1, t
        const unsigned char* s0m = ring0 + (size_t)((k0 + j - 2) % FD0) * p.slot0;
        const unsigned char* s0c = ring0 + (size_t)((k0 + j - 1) % FD0) * p.slot0;
        const unsigned char* s0p = ring0 + (size_t)((k0 + j) % FD0) * p.slot0;
        const unsigned char* s1c = ring1 + (size_t)((k1 + j) % FD1) * p.slot1;
        const int zq = wrap(t - 1, L);
#pragma unroll
        for (int k = 0; k < FMAXI; ++k) {
          if (rba[k] < 0) continue;
          const int r = rba[k], xh = xba[k];
          const int o = (f.y0 + r + t) & 1;
          const int r0 = r + f.hp0, r1 = r + f.hp1;
          int xp = xh + o, xm = xh + o - 1;
          if (xp == Lh) xp = 0;
          if (xm < 0) xm = Lh - 1;
          int ryp = r0 + 1, rym = r0 - 1;
          if (f.full) {
            if (ryp == L) ryp = 0;
            if (rym < 0) rym = L - 1;
          }
          Chunk nc[6][PL];
          lds_chunks<F>(s0c + r0 * RB + xp * CH, pb0, nc[0]);
          lds_chunks<F>(s0c + r0 * RB + xm * CH, pb0, nc[1]);
          lds_chunks<F>(s0c + ryp * RB + xh * CH, pb0, nc[2]);
          lds_chunks<F>(s0c + rym * RB + xh * CH, pb0, nc[3]);
          lds_chunks<F>(s0p + r0 * RB + xh * CH, pb0, nc[4]);
          lds_chunks<F>(s0m + r0 * RB + xh * CH, pb0, nc[5]);
          Chunk c[PL];
          lds_chunks<F>(s1c + r1 * RB + xh * CH, pb1, c);
          or_chunk<F, J16>(nc, c, rc1[k]);
          const long long ss = half + (long long)Lh * (f.y0 + r + (long long)L * zq) + xh;
#pragma unroll
          for (int pl = 0; pl < PL; ++pl) *reinterpret_cast<Chunk*>(dstg + pl * ps + ss * CH) = c[pl];
        }
      }
      consumer_bar();
      if (*s_abort) {
        aborted = true;
        break;
      }
      if (ct == 0) {
        // slots released by this step: odd plane t-1 and even plane t-2 (all of
        // the item's remaining ones after its last step); refill them
        const uint32_t rel1 = k1 + j + (j < nsteps - 1 ? 1u : 3u);
        const uint32_t rel0 = j < nsteps - 1 ? (j >= 2 ? k0 + j - 1 : k0) : k0 + j + 1;
        advance<F>(p, c1, 1, rel1 + FD1, ring1, p.slot1, full1, FD1);
        advance<F>(p, c0, 0, rel0 + FD0, ring0, p.slot0, full0, FD0);
      }
    }
    k1 += nsteps + 2;
    k0 += nsteps;
  }
  if (ct == 0 && aborted) {
    // wind down: let the copies still in flight land before the block exits
    for (uint32_t k = c1.k > (uint32_t)FD1 ? c1.k - FD1 : 0u; k < c1.k; ++k)
      mbar_wait(full1 + k % FD1, (k / FD1) & 1u, p.timeout_ns);
    for (uint32_t k = c0.k > (uint32_t)FD0 ? c0.k - FD0 : 0u; k < c0.k; ++k)
      mbar_wait(full0 + k % FD0, (k / FD0) & 1u, p.timeout_ns);
  }
}

template <int F>
static cudaError_t launch_f(bool j16, const FusedParams& p, int grid, size_t smem, cudaStream_t st) {
  if (j16) {
    k_fused_or<F, true><<<grid, FNCT, smem, st>>>(p);
  } else {
    k_fused_or<F, false><<<grid, FNCT, smem, st>>>(p);
  }
  return cudaGetLastError();
}

template <int F>
static cudaError_t prepare_f(bool j16, size_t smem, int* per_sm) {
  const void* fn = j16 ? (const void*)k_fused_or<F, true> : (const void*)k_fused_or<F, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, FNCT, smem);
}

cudaError_t prepare_fused(int fmt, bool j16, size_t smem, int* blocks_per_sm) {
  switch (fmt) {
    case FMT_F32: return prepare_f<FMT_F32>(j16, smem, blocks_per_sm);
    case FMT_F16: return prepare_f<FMT_F16>(j16, smem, blocks_per_sm);
    case FMT_BF16: return prepare_f<FMT_BF16>(j16, smem, blocks_per_sm);
    case FMT_ANG16: return prepare_f<FMT_ANG16>(j16, smem, blocks_per_sm);
    case FMT_OCT16: return prepare_f<FMT_OCT16>(j16, smem, blocks_per_sm);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused(int fmt, bool j16, const FusedParams& p, int grid, size_t smem,
                         cudaStream_t st) {
  if (grid <= 0 || p.n_items <= 0) return cudaSuccess;
  switch (fmt) {
    case FMT_F32: return launch_f<FMT_F32>(j16, p, grid, smem, st);
    case FMT_F16: return launch_f<FMT_F16>(j16, p, grid, smem, st);
    case FMT_BF16: return launch_f<FMT_BF16>(j16, p, grid, smem, st);
    case FMT_ANG16: return launch_f<FMT_ANG16>(j16, p, grid, smem, st);
    case FMT_OCT16: return launch_f<FMT_OCT16>(j16, p, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hsg
