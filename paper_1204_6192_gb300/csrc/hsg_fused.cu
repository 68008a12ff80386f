// Fused over-relaxation sweep: both half-sweeps of the double checkerboard
// (Sec. 3.1, Eq. 3) in one launch, every spin read once and written once.
//
// A block walks a column of the lattice -- one chunk group (4 systems) of one
// sample, a band of ny rows of y (all x), a range of planes [za, zb) -- as a
// wavefront along z.  In the step at plane t it updates the even sites of plane
// t (from the odd sites of planes t-1, t, t+1, all still old) and the odd sites
// of plane t-2 (from the even sites of planes t-3, t-2, t-1, all updated in
// earlier steps).  The two sets do not depend on each other, so one block
// barrier per step suffices, and every thread gets the same number of sites.
// That is the order of the two half-sweeps: every even site sees only old odd
// spins and every odd site only new even spins, so the result equals the even
// half-sweep followed by the odd one, bit for bit (the same arithmetic in the
// same order as the per-half-sweep kernel).
//
// The sweep reads one spin buffer and writes the other, so blocks never wait
// for one another: the even sites a band's odd rows need from its neighbours
// (rows y0-1 and y0+ny) and those a segment needs from the planes beyond it
// (za-1 and zb) are recomputed from the old spins.  Odd and even spins reach
// shared memory by bulk copies (cp.async.bulk) into two rings of plane slots
// (odd: 6, even: 5), each with a full mbarrier.  One thread per ring (warps 0
// and 1) issues its copies: the first ones at the start, then, after every
// step, into the slots that step released (the threads are past the block
// barrier there), running ahead into the block's next work item.  The six bonds and the field of a site
// (shared by all chunk groups, so mostly L2 hits) are loaded one step ahead.
// Every wait is bounded: one that runs out sets the error word and the block
// winds down after its copies have landed.
#include <type_traits>

#include "hsg_async.cuh"
#include "hsg_device.cuh"
#include "hsg_internal.h"

namespace hsg {

namespace {

constexpr int FD1 = FUSED_ODD_SLOTS;    // odd-site plane slots
constexpr int FD0 = FUSED_EVEN_SLOTS;   // even-site plane slots
constexpr int FCW = FUSED_CONSUMER_WARPS;
constexpr int FNCT = FCW * 32;  // consumer threads
constexpr int FMAXI = FUSED_SITES_PER_THREAD;   // sites per thread and step (host-checked)
constexpr int FUSED_CURSOR_OFFSET = 128;         // the two copy cursors in the shared-memory head

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
// consumer: one site update from chunks in shared memory
// ---------------------------------------------------------------------------
template <bool J16>
struct Rec {
  // FP16 records: the 12 halves as three 8-byte words; FP32: three float4
  typename std::conditional<J16, uint2, float4>::type w[3];
};
static_assert(sizeof(Rec<true>) == 24 && sizeof(Rec<false>) == 48, "one record per storage site");

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
#pragma unroll
  for (int k = 0; k < VEC / 2; ++k) or_move2(s.x[k], s.y[k], s.z[k], hf.x[k], hf.y[k], hf.z[k]);
  encode<F>(s, c);
}

}  // namespace

// The queue of bulk copies of one ring: the odd-plane loads of every item of
// the block (planes za-2 .. zb+1; warp 0 issues them) or its even-plane loads
// (za-1 .. zb; warp 1), each issued as soon as a slot of its ring has been
// released, running into the next item.  The cursor keeps the current item's
// copy geometry, so a copy costs a few integer operations.
struct CopyCursor {
  int it;                    // current item (>= n_items: done)
  int m, n;                  // next load within the item, loads in the item (0: not decoded)
  uint32_t k;                // loads issued
  int q, L;                  // plane of the next load (wrapped), lattice size
  const unsigned char* src;  // component 0 of row ya of plane 0 of the ring's parity
  long long plane_stride;    // bytes between components
  long long plane_bytes;     // bytes between planes (Lh L CHUNK)
  long long wrap_back;       // bytes from row ya back to row 0 (second segment)
  uint32_t seg1, seg2;       // bytes of the two row segments (seg2 = 0: one segment)
  uint32_t slot_stride;      // bytes between components in the slot (R rows)
};

template <int F>
__device__ __forceinline__ void advance(const FusedParams& p, CopyCursor& c, int parity, uint32_t limit,
                                        unsigned char* ring, uint32_t slot_bytes, uint64_t* full,
                                        uint32_t D) {
  constexpr int CH = FmtInfo<F>::CHUNK, PL = FmtInfo<F>::PLANES;
  while (c.k < limit && c.it < p.n_items) {
    if (c.n == 0) {
      // decode the item once
      const FItem f = item_geom(p, c.it);
      if (!p.active[f.s]) {
        c.it += gridDim.x;
        continue;
      }
      const SampleDev& sd = p.samples[f.s];
      const int L = f.L, R = parity ? f.R1 : f.R0;
      const int ya = wrap(f.y0 - (parity ? f.hp1 : f.hp0), L);
      const uint32_t RB = (uint32_t)f.Lh * CH;
      const int n1 = min(R, L - ya);
      c.n = f.zb - f.za + (parity ? 4 : 2);
      c.m = 0;
      c.L = L;
      c.q = ((parity ? f.za - 2 : f.za - 1) + L) % L;
      c.plane_stride = sd.plane_stride;
      c.plane_bytes = (long long)f.Lh * L * CH;
      c.src = p.src + sd.spin_off + (long long)f.g * sd.N * CH +
              ((long long)parity * (sd.N >> 1) + (long long)f.Lh * ya) * CH;
      c.wrap_back = (long long)f.Lh * ya * CH;
      c.seg1 = (uint32_t)n1 * RB;
      c.seg2 = (uint32_t)(R - n1) * RB;
      c.slot_stride = (uint32_t)R * RB;
    }
    unsigned char* slot = ring + (size_t)(c.k % D) * slot_bytes;
    uint64_t* bar = full + c.k % D;
    mbar_expect_tx(bar, (uint32_t)PL * (c.seg1 + c.seg2));
    const unsigned char* g = c.src + c.q * c.plane_bytes;
#pragma unroll
    for (int pl = 0; pl < PL; ++pl) {
      unsigned char* d = slot + pl * c.slot_stride;
      bulk_copy_g2s(d, g + pl * c.plane_stride, c.seg1, bar);
      if (c.seg2) bulk_copy_g2s(d + c.seg1, g + pl * c.plane_stride - c.wrap_back, c.seg2, bar);
    }
    ++c.k;
    if (++c.q == c.L) c.q = 0;
    if (++c.m == c.n) {
      c.it += gridDim.x;
      c.n = 0;
    }
  }
}

// One of a thread's sites in the current item (fixed for the whole item; the
// plane changes from step to step).
struct FSite {
  int kind;                 // -1: none, 0: even site, 1: odd site
  uint32_t own;             // byte offset of its chunk in its own slot (component 0)
  uint32_t xo[2], xm[2];    // byte offsets of its +x and -x neighbours (site x parity 0, 1)
  uint32_t yp, ym, zc;      // ... of its +y, -y neighbours and of itself in the z-neighbour slots
  int pb;                   // x parity of the site at plane t: (pb + t) & 1
  long long ss;             // storage site without the plane term
  bool out;                 // even sites: the row is the block's own (written out)
};

static_assert((FD1 + FD0) * 8 + 4 <= FUSED_CURSOR_OFFSET, "mbarriers overlap the copy cursors");
static_assert(FUSED_CURSOR_OFFSET + 2 * sizeof(CopyCursor) <= FUSED_SMEM_HEAD, "copy cursors overlap the rings");

template <int F, bool J16>
__global__ void __launch_bounds__(FNCT, 1) k_fused_or(const FusedParams p) {
  constexpr int CH = FmtInfo<F>::CHUNK, PL = FmtInfo<F>::PLANES;
  using Chunk = typename FmtInfo<F>::Chunk;
  using RecT = Rec<J16>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full1 = reinterpret_cast<uint64_t*>(smem);
  uint64_t* full0 = full1 + FD1;
  volatile int* s_abort = reinterpret_cast<volatile int*>(full0 + FD0);
  unsigned char* ring1 = smem + FUSED_SMEM_HEAD;
  unsigned char* ring0 = ring1 + (size_t)FD1 * p.slot1;
  const int ct = threadIdx.x;
  // copy cursors (in shared memory: only their two threads use them): odd
  // planes issued by thread 0, even planes by thread 32
  const bool issue1 = ct == 0, issue0 = ct == 32;
  CopyCursor& cc = reinterpret_cast<CopyCursor*>(smem + FUSED_CURSOR_OFFSET)[issue1 ? 0 : 1];
  if (issue1 || issue0) {
    cc.it = (int)blockIdx.x;
    cc.n = 0;
    cc.k = 0u;
  }
  if (ct == 0) {
    for (int k = 0; k < FD1; ++k) mbar_init(full1 + k, 1);
    for (int k = 0; k < FD0; ++k) mbar_init(full0 + k, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (issue1) advance<F>(p, cc, 1, FD1, ring1, p.slot1, full1, FD1);
  if (issue0) advance<F>(p, cc, 0, FD0, ring0, p.slot0, full0, FD0);

  uint32_t k1 = 0, k0 = 0;   // loads consumed (and released) before the current item
  bool aborted = false;
  for (int it = blockIdx.x; it < p.n_items && !aborted; it += gridDim.x) {
    const FItem f = item_geom(p, it);
    if (!p.active[f.s]) continue;
    const SampleDev& sd = p.samples[f.s];
    const int L = f.L, Lh = f.Lh;
    const int nsteps = f.zb - f.za + 3;
    const uint32_t RB = (uint32_t)Lh * CH;
    const uint32_t pb1 = (uint32_t)f.R1 * RB, pb0 = (uint32_t)f.R0 * RB;
    const int nP0 = f.R0 * Lh, nP1 = f.ny * Lh;
    const long long ps = sd.plane_stride;
    unsigned char* dstg = p.dst + sd.spin_off + (long long)f.g * sd.N * CH;
    const long long rbase = sd.rec_off;
    const long long plane_sites = (long long)Lh * L;
    // this thread's sites: the even sites of the slot rows first, then the odd
    // sites of the band rows
    FSite st[FMAXI];
#pragma unroll
    for (int k = 0; k < FMAXI; ++k) {
      int i = ct + k * FNCT;
      FSite& q = st[k];
      q.kind = i < nP0 ? 0 : (i < nP0 + nP1 ? 1 : -1);
      if (q.kind == 1) i -= nP0;
      const int rr = (int)((__umulhi((uint32_t)i, sd.fdLh_m) + (uint32_t)i) >> sd.fdLh_s);
      const int xh = i - rr * Lh;
      // rown: the site's row in the slots it reads (odd slots for even sites and
      // vice versa); rowo: its row in its own slot
      const int rown = q.kind == 0 ? rr + (f.hp1 - f.hp0) : rr + f.hp0;
      const int rowo = q.kind == 0 ? rr : rr + f.hp1;
      int ryp = rown + 1, rym = rown - 1;
      if (f.full) {
        if (ryp == L) ryp = 0;
        if (rym < 0) rym = L - 1;
      }
      q.own = (uint32_t)rowo * RB + (uint32_t)xh * CH;
      q.zc = (uint32_t)rown * RB + (uint32_t)xh * CH;
      q.yp = (uint32_t)ryp * RB + (uint32_t)xh * CH;
      q.ym = (uint32_t)rym * RB + (uint32_t)xh * CH;
#pragma unroll
      for (int o = 0; o < 2; ++o) {
        // x = 2 xh + o: the +x neighbour has half-x xh + o, the -x neighbour xh + o - 1
        const int xp = xh + o == Lh ? 0 : xh + o;
        const int xm = xh + o - 1 < 0 ? Lh - 1 : xh + o - 1;
        q.xo[o] = (uint32_t)rown * RB + (uint32_t)xp * CH;
        q.xm[o] = (uint32_t)rown * RB + (uint32_t)xm * CH;
      }
      const int y = q.kind == 0 ? wrap(f.y0 - f.hp0 + rr, L) : f.y0 + rr;
      // x = 2 xh + ((y + z + parity) & 1); the odd sites sit on plane t - 2
      q.pb = q.kind == 0 ? y : y - 1;
      q.out = q.kind == 0 && rr >= f.hp0 && rr < f.hp0 + f.ny;
      q.ss = (q.kind == 1 ? (sd.N >> 1) : 0) + (long long)Lh * y + xh;
    }
    // planes of the step (wrapped): t for the even sites, t - 2 for the odd ones
    int z0 = wrap(f.za - 1, L), z1 = wrap(f.za - 3 + L, L);
    // ring slots, rotated one plane per step: odd planes t-2 (own of the odd
    // sites), t-1, t, t+1; even planes t-3, t-2, t-1 and t (own of the even sites)
    uint32_t i1 = (k1 + 2) % FD1, ph1 = ((k1 + 2) / FD1) & 1u;   // slot, phase of odd plane t+1
    uint32_t i0 = k0 % FD0, ph0 = (k0 / FD0) & 1u;               // slot, phase of even plane t
    const unsigned char* o_own = ring1;
    const unsigned char* o_m = ring1 + (size_t)(k1 % FD1) * p.slot1;
    const unsigned char* o_c = ring1 + (size_t)((k1 + 1) % FD1) * p.slot1;
    const unsigned char* o_p = ring1 + (size_t)i1 * p.slot1;
    const unsigned char* e_m = ring0;
    const unsigned char* e_c = ring0;
    const unsigned char* e_p = ring0;
    unsigned char* e_t = ring0 + (size_t)i0 * p.slot0;
    RecT rc[FMAXI], rn[FMAXI];
    // couplings and field of the sites of a step (even sites on plane za, odd on za-2 ... )
#pragma unroll
    for (int k = 0; k < FMAXI; ++k)
      if (st[k].kind == 0) load_rec<J16>(p.rec, rbase + st[k].ss + plane_sites * z0, rn[k]);
    for (int j = 0; j < nsteps; ++j) {
      const int t = f.za - 1 + j;
      const bool do0 = t <= f.zb, do1 = t - 2 >= f.za;
#pragma unroll
      for (int k = 0; k < FMAXI; ++k) rc[k] = rn[k];
      const int zn0 = z0 + 1 == L ? 0 : z0 + 1, zn1 = z1 + 1 == L ? 0 : z1 + 1;
      if (j + 1 < nsteps) {
        // next step's records: even sites on plane t + 1, odd sites on plane t - 1
        const long long a0 = plane_sites * zn0, a1 = plane_sites * zn1;
#pragma unroll
        for (int k = 0; k < FMAXI; ++k) {
          if (st[k].kind == 0 && t + 1 <= f.zb) load_rec<J16>(p.rec, rbase + st[k].ss + a0, rn[k]);
          if (st[k].kind == 1 && t - 1 >= f.za) load_rec<J16>(p.rec, rbase + st[k].ss + a1, rn[k]);
        }
      }
      bool ok = true;
      if (do0) {
        if (j == 0) {
          for (uint32_t m = 0; m < 2; ++m)
            ok = ok && mbar_wait(full1 + (k1 + m) % FD1, ((k1 + m) / FD1) & 1u, p.timeout_ns);
        }
        ok = ok && mbar_wait(full1 + i1, ph1, p.timeout_ns);
        ok = ok && mbar_wait(full0 + i0, ph0, p.timeout_ns);
      }
      if (!ok) {
        atomicOr(p.err, 1u);
        *s_abort = 1;
      }
      if (!*s_abort) {
        const long long d0 = plane_sites * z0, d1 = plane_sites * z1;
        const bool write0 = t >= f.za && t < f.zb;
#pragma unroll
        for (int k = 0; k < FMAXI; ++k) {
          const FSite& q = st[k];
          const bool even = q.kind == 0;
          if (even ? !do0 : (q.kind != 1 || !do1)) continue;
          const int o = (q.pb + t) & 1;
          const unsigned char* nc_ = even ? o_c : e_c;   // same plane
          const unsigned char* np_ = even ? o_p : e_p;   // + z
          const unsigned char* nm_ = even ? o_m : e_m;   // - z
          const uint32_t pbn = even ? pb1 : pb0, pbo = even ? pb0 : pb1;
          Chunk nc[6][PL];
          lds_chunks<F>(nc_ + (o ? q.xo[1] : q.xo[0]), pbn, nc[0]);
          lds_chunks<F>(nc_ + (o ? q.xm[1] : q.xm[0]), pbn, nc[1]);
          lds_chunks<F>(nc_ + q.yp, pbn, nc[2]);
          lds_chunks<F>(nc_ + q.ym, pbn, nc[3]);
          lds_chunks<F>(np_ + q.zc, pbn, nc[4]);
          lds_chunks<F>(nm_ + q.zc, pbn, nc[5]);
          unsigned char* own = (even ? e_t : const_cast<unsigned char*>(o_own)) + q.own;
          Chunk c[PL];
          lds_chunks<F>(own, pbo, c);
          or_chunk<F, J16>(nc, c, rc[k]);
          if (even) sts_chunks<F>(own, pb0, c);
          if (even ? (write0 && q.out) : true) {
            unsigned char* g = dstg + (q.ss + (even ? d0 : d1)) * CH;
#pragma unroll
            for (int pl = 0; pl < PL; ++pl) *reinterpret_cast<Chunk*>(g + pl * ps) = c[pl];
          }
        }
        // the even slot is refilled by bulk copies (async proxy) once released
        if (do0) fence_proxy_async_smem();
      }
      consumer_bar();
      if (*s_abort) {
        aborted = true;
        break;
      }
      // released by this step: odd plane t-2 and even plane t-3 (every slot of
      // the item after its last step); refill them
      if (issue1) {
        const uint32_t rel1 = k1 + (j == nsteps - 1 ? (uint32_t)nsteps + 1u : (uint32_t)j);
        advance<F>(p, cc, 1, rel1 + FD1, ring1, p.slot1, full1, FD1);
      }
      if (issue0) {
        const uint32_t rel0 = k0 + (j == nsteps - 1 ? (uint32_t)nsteps - 1u : (uint32_t)max(0, j - 2));
        advance<F>(p, cc, 0, rel0 + FD0, ring0, p.slot0, full0, FD0);
      }
      // next step: planes and slots move by one
      z0 = zn0;
      z1 = zn1;
      o_own = o_m;
      o_m = o_c;
      o_c = o_p;
      if (++i1 == FD1) {
        i1 = 0;
        ph1 ^= 1u;
      }
      o_p = ring1 + (size_t)i1 * p.slot1;
      e_m = e_c;
      e_c = e_p;
      e_p = e_t;
      if (++i0 == FD0) {
        i0 = 0;
        ph0 ^= 1u;
      }
      e_t = ring0 + (size_t)i0 * p.slot0;
    }
    k1 += nsteps + 1;
    k0 += nsteps - 1;
  }
  if (aborted && (issue1 || issue0)) {
    // wind down: let the copies still in flight land before the block exits
    const uint32_t D = issue1 ? FD1 : FD0;
    uint64_t* full = issue1 ? full1 : full0;
    for (uint32_t k = cc.k > D ? cc.k - D : 0u; k < cc.k; ++k)
      mbar_wait(full + k % D, (k / D) & 1u, p.timeout_ns);
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
