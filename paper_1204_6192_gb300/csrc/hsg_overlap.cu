// Replica-pair measurements (Sec. 2 of the paper's observables): the overlap
// tensor q^{mu nu}(k) of replicas 0 and 1 (Eq. 5 and its k-dependent form),
// the scalar pair overlaps D_ab(k) that the four-replica sums chi_1, chi_2,
// chi_3 are built from, and the chiral overlaps C_ab^alpha(k) of the local
// chirality kappa_i^alpha = s_{i+alpha} . (s_i x s_{i-alpha}).  Modes
// k = 0 and (2 pi / L) e_x, e_y, e_z, sign e^{+i k.R}.
//
// For a slot t and pair (a, b), A and B are the configurations replicas a and
// b hold at t.  The four-replica sums contract the spin components within each
// site, so chi_1 = N^2 |D_12|^2, chi_2 = N^2 D_13 conj(D_14),
// chi_3 = N^2 D_13 conj(D_24) (replicas numbered from 1); the host assembles them.
//
// A block covers a tile of MEAS_TILE consecutive sites of one sample (and one
// pair) for every slot: each warp takes one slot at a time and walks the tile
// in runs of 32 consecutive sites, so a spin load of the warp is contiguous
// within each parity half, and the four systems of a storage chunk, which
// belong to different slots, meet the tile's lines in L1 or L2.  A thread sums
// its sites of the tile per slot in FP32 (loading several sites' spins before
// using any, for memory-level parallelism), the warp adds its lanes in FP32 and writes
// one FP64 partial per (tile, slot); the final kernel adds the tiles in FP64 in
// a fixed order.  (GB300's FP64 rate is a small fraction of its FP32 rate, so FP64
// work is kept per tile, not per site.)  These direct kernels serve the chiral
// overlaps, whose neighbours lie outside any run of storage sites, and
// contexts whose staged systems do not fit shared memory.
//
// The staged kernels (tensor q(k) and scalar D_ab(k)) read each spin once: a
// block owns a run of consecutive storage sites of one sample (both parity
// halves are such runs, and a site's coordinates follow from its index).  Its
// thread 0 brings the spins of the measured replicas into shared memory with
// bulk asynchronous copies (one contiguous copy per plane and chunk group),
// `sub` sites per stage and three stages in flight, each completing on its
// own mbarrier.  The lanes of a warp are slots: lane t decodes, from shared
// memory, the spins its replicas hold at slot t (memory slots through perm),
// so one warp step covers one storage site for up to 32 slots (32 / TL sites
// for TL < 32 slots).  A lane keeps its slot's sums in FP32 over the block's
// run; the block adds its warps in FP32 in warp order and writes one FP64
// partial per (block, slot, value), which the final kernel adds in FP64 in a
// fixed order.  Every wait on a stage is bounded by the context's barrier timeout;
// one that runs out sets the error word, which the host reports.
#include "hsg_async.cuh"
#include "hsg_kernels.cuh"

namespace hsg {

namespace {

// replica pairs in the order (0,1) (0,2) (1,2) (0,3) (1,3) (2,3): the pairs of
// the first r replicas come first
__device__ __forceinline__ void pair_of(int k, int& a, int& b) {
  const int A[6] = {0, 0, 1, 0, 1, 2}, B[6] = {1, 2, 2, 3, 3, 3};
  a = A[k];
  b = B[k];
}

struct V3 {
  float x, y, z;
};

__device__ __forceinline__ float dot3(const V3& a, const V3& b) {
  return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x)));
}

// a . (b x c)
__device__ __forceinline__ float triple(const V3& a, const V3& b, const V3& c) {
  const float cx = __fsub_rn(__fmul_rn(b.y, c.z), __fmul_rn(b.z, c.y));
  const float cy = __fsub_rn(__fmul_rn(b.z, c.x), __fmul_rn(b.x, c.z));
  const float cz = __fsub_rn(__fmul_rn(b.x, c.y), __fmul_rn(b.y, c.x));
  return __fmaf_rn(a.z, cz, __fmaf_rn(a.y, cy, __fmul_rn(a.x, cx)));
}

template <int F>
__device__ __forceinline__ V3 spin_at(const unsigned char* base, const SampleDev& sd, int w, int L,
                                      int x, int y, int z) {
  const uint32_t site = (uint32_t)x + (uint32_t)L * ((uint32_t)y + (uint32_t)L * (uint32_t)z);
  const uint32_t ss = (((uint32_t)(x + y + z)) & 1u) * ((uint32_t)sd.N >> 1) + (site >> 1);
  V3 v;
  decode_one<F>(base + chunk_offset<F>(sd, (uint32_t)w >> 2, ss), sd.plane_stride, w & 3, v.x, v.y,
                v.z);
  return v;
}

constexpr int NM = 7;        // per product: k = 0, then (re, im) of kx, ky, kz

// what a launch measures
enum { MEAS_QTENSOR = 0, MEAS_PAIRS = 1, MEAS_PAIRS_CHIRAL = 2, MEAS_CHIRAL = 3 };

// products per site of one launch unit: a row mu of the tensor (A^mu B^nu,
// nu = x, y, z; three units), or D (and C^x, C^y, C^z) of one pair
template <int MODE>
__host__ __device__ constexpr int n_products() {
  return MODE == MEAS_QTENSOR ? 3 : (MODE == MEAS_PAIRS ? 1 : 4);
}

}  // namespace

template <int F, int MODE>
__global__ void __launch_bounds__(MEAS_BS) k_meas_tiles(const OverlapParams p) {
  constexpr int NP = n_products<MODE>();
  constexpr int NVAL = NP * NM;
  // units of one tile are consecutive blocks, so they meet the tile's lines in L2
  const int s = blockIdx.y, unit = blockIdx.x % p.n_pairs, tile = blockIdx.x / p.n_pairs;
  const SampleDev& sd = p.samples[s];
  const int L = sd.L, R_T = p.R_T;
  const uint32_t N = (uint32_t)sd.N;
  const uint32_t i_begin = tile * MEAS_TILE;
  if (i_begin >= N) return;
  const uint32_t i_end = min(N, i_begin + (uint32_t)MEAS_TILE);
  __shared__ float tw[2][512];
  for (int x = threadIdx.x; x < L; x += blockDim.x) {
    float sx, cx;
    sincospif(2.0f * (float)x / (float)L, &sx, &cx);
    tw[0][x] = cx;
    tw[1][x] = sx;
  }
  __syncthreads();
  int a = 0, b = 1;
  if (MODE != MEAS_QTENSOR) pair_of(unit, a, b);
  const int* perm = p.perm + (long long)s * p.R_O * R_T;
  const unsigned char* base = p.spins + sd.spin_off;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* out = p.partials + (((long long)s * p.n_pairs + unit) * p.n_tiles + tile) * R_T * NVAL;
  // each warp takes one slot at a time and walks the tile in runs of 32 sites
  for (int t = warp; t < R_T; t += MEAS_BS / 32) {
    const int wA = a * R_T + perm[a * R_T + t], wB = b * R_T + perm[b * R_T + t];
    float acc[NVAL];
#pragma unroll
    for (int k = 0; k < NVAL; ++k) acc[k] = 0.0f;
    // U sites per thread per round, all their spins loaded before any is used
    constexpr int U = MODE == MEAS_PAIRS_CHIRAL ? 2 : 4;
    for (uint32_t i0 = i_begin + lane; i0 < i_end; i0 += 32 * U) {
      int xs[U], ys[U], zs[U];
      bool ok[U];
      V3 A[U], B[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = i0 + 32u * u;
        ok[u] = i < i_end;
        const uint32_t ic = ok[u] ? i : i_begin;
        const uint32_t r = (__umulhi(ic, sd.fdL_m) + ic) >> sd.fdL_s;     // i / L
        const uint32_t zz = (__umulhi(r, sd.fdL_m) + r) >> sd.fdL_s;      // r / L
        xs[u] = (int)(ic - r * (uint32_t)L);
        ys[u] = (int)(r - zz * (uint32_t)L);
        zs[u] = (int)zz;
        A[u] = spin_at<F>(base, sd, wA, L, xs[u], ys[u], zs[u]);
        B[u] = spin_at<F>(base, sd, wB, L, xs[u], ys[u], zs[u]);
      }
      float kap[U][3][2];
      if constexpr (MODE == MEAS_PAIRS_CHIRAL) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int x = xs[u], y = ys[u], z = zs[u];
          const int xp = (x + 1 == L) ? 0 : x + 1, xm = (x == 0) ? L - 1 : x - 1;
          const int yp = (y + 1 == L) ? 0 : y + 1, ym = (y == 0) ? L - 1 : y - 1;
          const int zp = (z + 1 == L) ? 0 : z + 1, zm = (z == 0) ? L - 1 : z - 1;
          kap[u][0][0] = triple(spin_at<F>(base, sd, wA, L, xp, y, z), A[u], spin_at<F>(base, sd, wA, L, xm, y, z));
          kap[u][0][1] = triple(spin_at<F>(base, sd, wB, L, xp, y, z), B[u], spin_at<F>(base, sd, wB, L, xm, y, z));
          kap[u][1][0] = triple(spin_at<F>(base, sd, wA, L, x, yp, z), A[u], spin_at<F>(base, sd, wA, L, x, ym, z));
          kap[u][1][1] = triple(spin_at<F>(base, sd, wB, L, x, yp, z), B[u], spin_at<F>(base, sd, wB, L, x, ym, z));
          kap[u][2][0] = triple(spin_at<F>(base, sd, wA, L, x, y, zp), A[u], spin_at<F>(base, sd, wA, L, x, y, zm));
          kap[u][2][1] = triple(spin_at<F>(base, sd, wB, L, x, y, zp), B[u], spin_at<F>(base, sd, wB, L, x, y, zm));
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (!ok[u]) continue;
        float P[NP];
        if constexpr (MODE == MEAS_QTENSOR) {
          const float am = unit == 0 ? A[u].x : (unit == 1 ? A[u].y : A[u].z);   // unit = mu
          P[0] = __fmul_rn(am, B[u].x);
          P[1] = __fmul_rn(am, B[u].y);
          P[2] = __fmul_rn(am, B[u].z);
        } else {
          P[0] = dot3(A[u], B[u]);
          if constexpr (MODE == MEAS_PAIRS_CHIRAL) {
#pragma unroll
            for (int d = 0; d < 3; ++d) P[1 + d] = __fmul_rn(kap[u][d][0], kap[u][d][1]);
          }
        }
        const int x = xs[u], y = ys[u], z = zs[u];
        const float c3[3] = {tw[0][x], tw[0][y], tw[0][z]}, s3[3] = {tw[1][x], tw[1][y], tw[1][z]};
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          acc[q * NM] = __fadd_rn(acc[q * NM], P[q]);
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            acc[q * NM + 1 + 2 * d] = __fmaf_rn(P[q], c3[d], acc[q * NM + 1 + 2 * d]);
            acc[q * NM + 2 + 2 * d] = __fmaf_rn(P[q], s3[d], acc[q * NM + 2 + 2 * d]);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NVAL; ++k) {
      const float w = warp_sum(acc[k]);
      if (lane == 0) out[(long long)t * NVAL + k] = (double)w;
    }
  }
}

// One warp per (sample, unit, slot, value): lane l adds the tiles' partials
// l, l + 32, ... in that order, then the lanes are added in a fixed butterfly;
// the total times 1/N.  Eight values per block of 256 threads.
template <int MODE>
__global__ void __launch_bounds__(256) k_meas_final(const OverlapParams p) {
  constexpr int NP = n_products<MODE>();
  constexpr int NVAL = NP * NM;
  const int t = blockIdx.x % p.R_T, su = blockIdx.x / p.R_T;
  const int unit = su % p.n_pairs, s = su / p.n_pairs;
  const int v = blockIdx.y * 8 + (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (v >= NVAL) return;
  const SampleDev& sd = p.samples[s];
  const int n_tiles = (int)(((long long)sd.N + MEAS_TILE - 1) / MEAS_TILE);
  const long long stride = (long long)p.R_T * NVAL;
  const double* src = p.partials + ((long long)s * p.n_pairs + unit) * p.n_tiles * stride +
                      (long long)t * NVAL + v;
  double sum = 0.0;
#pragma unroll 4
  for (int k = lane; k < n_tiles; k += 32) sum += src[k * stride];
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane != 0) return;
  const double val = sum / (double)sd.N;
  const int q = v / NM, m = v % NM;
  if constexpr (MODE == MEAS_QTENSOR) {
    const int mn = unit * 3 + q;     // mu * 3 + nu
    if (m == 0) {
      if (p.D) p.D[((long long)s * p.R_T + t) * 9 + mn] = val;
    } else if (p.C) {
      const int d = (m - 1) / 2, ri = (m - 1) % 2;
      p.C[(((long long)s * p.R_T + t) * 3 + d) * 18 + mn * 2 + ri] = val;
    }
  } else {
    const int mode = m == 0 ? 0 : 1 + (m - 1) / 2, ri = m == 0 ? 0 : (m - 1) % 2;
    double* dst = nullptr;
    if (q == 0) dst = p.D ? p.D + (((long long)s * p.R_T + t) * p.n_pairs + unit) * 8 : nullptr;
    else dst = p.C ? p.C + ((((long long)s * p.R_T + t) * p.n_pairs + unit) * 3 + (q - 1)) * 8 : nullptr;
    if (dst) {
      dst[2 * mode + ri] = val;
      if (m == 0) dst[1] = 0.0;
    }
  }
}

// ---------------------------------------------------------------------------
// Staged kernels
// ---------------------------------------------------------------------------
namespace {

constexpr int MS_STAGES = 3;   // stages in flight per block

// products per site: the nine A^mu B^nu of replicas 0 and 1, or the pair dot
// products of NR replicas
template <int MODE, int NR>
__host__ __device__ constexpr int staged_products() {
  return MODE == MEAS_QTENSOR ? 9 : (MODE == MEAS_CHIRAL ? 3 : 1) * (NR * (NR - 1) / 2);
}

}  // namespace

template <int F, int MODE, int NR>
__global__ void __launch_bounds__(MEAS_BS) k_meas_staged(const OverlapParams p) {
  using FI = FmtInfo<F>;
  constexpr int NQ = staged_products<MODE, NR>();
  constexpr int NV = NQ * NM;
  constexpr int NW = MEAS_BS / 32;
  extern __shared__ __align__(128) unsigned char stage[];
  __shared__ uint64_t full[MS_STAGES];   // a stage's copies have landed
  __shared__ uint64_t empty[MS_STAGES];  // every warp is done with a stage's buffer
  __shared__ float2 tw[512];             // (cos, sin)(2 pi x / L)
  __shared__ float red[NV][32];          // the block's sums per (value, slot of the round)
  const int s = blockIdx.z, round = blockIdx.y;
  // the sample's geometry in registers: the loop's barrier operations are
  // memory clobbers, which would otherwise reload it every site
  const SampleDev sd = p.samples[s];
  const uint32_t N = (uint32_t)sd.N, Nh = N >> 1;
  const uint32_t b0 = blockIdx.x * (uint32_t)p.tile_ss;
  if (b0 >= N) return;
  const uint32_t b1 = min(N, b0 + (uint32_t)p.tile_ss);
  const int sub = p.sub;
  const int n_sub = (int)((b1 - b0 + (uint32_t)sub - 1) / (uint32_t)sub);
  const long long PS = (long long)p.Gu * p.grow;           // shared bytes between planes
  const int stage_bytes = FI::PLANES * (int)PS;
  const unsigned char* gsp = p.spins + sd.spin_off;
  const int L = sd.L, R_T = p.R_T;

  if (threadIdx.x == 0) {
    for (int k = 0; k < MS_STAGES; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], NW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int x = threadIdx.x; x < L; x += blockDim.x) {
    float sn, cs;
    sincospif(2.0f * (float)x / (float)L, &sn, &cs);
    tw[x] = make_float2(cs, sn);
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // stage k of the run: sub-run k into buffer k % MS_STAGES, one copy per
  // (plane, chunk group) row, issued by the lanes of warp 0 after lane 0 has
  // announced the stage's bytes
  const int rows = FI::PLANES * p.Gu;
  auto issue = [&](int k) {
    const int b = k % MS_STAGES;
    const uint32_t ss0 = b0 + (uint32_t)k * (uint32_t)sub;
    const uint32_t bytes = min((uint32_t)sub, b1 - ss0) * (uint32_t)FI::CHUNK;
    if (lane == 0) mbar_expect_tx(&full[b], bytes * (uint32_t)rows);
    __syncwarp();
    unsigned char* dst = stage + b * stage_bytes;
    for (int row = lane; row < rows; row += 32) {
      const int pl = row / p.Gu, g = row - pl * p.Gu;
      bulk_copy_g2s(dst + pl * PS + (long long)g * p.grow,
                    gsp + pl * sd.plane_stride + ((long long)g * N + ss0) * FI::CHUNK, bytes, &full[b]);
    }
  };
  int issued = min(MS_STAGES, n_sub);   // stages issued so far (warp 0)
  if (warp == 0)
    for (int k = 0; k < issued; ++k) issue(k);

  // lanes: TL slots per site group, 32 / TL site groups per warp
  const int nt = min(32, R_T - 32 * round);
  int TL = 1;
  while (TL < nt) TL <<= 1;
  const int tl = lane & (TL - 1), grp = lane / TL, SPW = 32 / TL;
  const bool live = tl < nt;
  const int t = 32 * round + tl;
  int off[NR], jw[NR];
  const int* perm = p.perm + (long long)s * p.R_O * R_T;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int w = live ? r * R_T + perm[r * R_T + t] : 0;
    off[r] = (w >> 2) * p.grow;
    jw[r] = w & 3;
  }
  float a0[NQ];
  float2 ak[NQ][3];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    a0[q] = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) ak[q][d] = make_float2(0.0f, 0.0f);
  }

  // No block-wide barrier in the loop: a warp waits for a stage's copies
  // (full) and, after its sites, arrives on the stage's empty barrier; warp 0
  // refills a buffer once every warp has arrived.  Decisions on a wait that
  // ran out are taken per warp, so a warp leaves the loop as a whole.
  bool ok = true;
  int k = 0;
  for (; k < n_sub; ++k) {
    const int b = k % MS_STAGES;
    const uint32_t ph = (uint32_t)(k / MS_STAGES) & 1u;
    if (!__all_sync(0xffffffffu, mbar_wait(&full[b], ph, p.timeout_ns))) {
      ok = false;
      break;
    }
    const uint32_t ss0 = b0 + (uint32_t)k * (uint32_t)sub;
    const int n = (int)min((uint32_t)sub, b1 - ss0);
    const unsigned char* st = stage + b * stage_bytes;
    for (int j = warp * SPW + grp; j < n; j += NW * SPW) {
      const uint32_t ss = ss0 + (uint32_t)j;
      const uint32_t par = ss >= Nh ? 1u : 0u;
      const uint32_t h = ss - par * Nh;                                  // site >> 1
      const uint32_t r = (__umulhi(h, sd.fdLh_m) + h) >> sd.fdLh_s;       // h / (L / 2)
      const uint32_t zz = (__umulhi(r, sd.fdL_m) + r) >> sd.fdL_s;        // r / L
      const uint32_t y = r - zz * (uint32_t)L;
      const uint32_t x = 2u * (h - r * (uint32_t)sd.Lh) + ((par + y + zz) & 1u);
      const float2 tk[3] = {tw[x], tw[y], tw[zz]};
      if (!live) continue;
      V3 S[NR];
#pragma unroll
      for (int rr = 0; rr < NR; ++rr)
        decode_one<F>(st + off[rr] + j * FI::CHUNK, PS, jw[rr], S[rr].x, S[rr].y, S[rr].z);
      float P[NQ];
      if constexpr (MODE == MEAS_QTENSOR) {
        const float A[3] = {S[0].x, S[0].y, S[0].z}, B[3] = {S[1].x, S[1].y, S[1].z};
#pragma unroll
        for (int mu = 0; mu < 3; ++mu)
#pragma unroll
          for (int nu = 0; nu < 3; ++nu) P[3 * mu + nu] = __fmul_rn(A[mu], B[nu]);
      } else if constexpr (MODE == MEAS_CHIRAL) {
        // the staged "spins" are the chiralities (kappa^x, kappa^y, kappa^z):
        // per pair, in the pair order below, the three products kappa^a kappa^b
        int q = 0;
#pragma unroll
        for (int bb = 1; bb < NR; ++bb)
#pragma unroll
          for (int aa = 0; aa < bb; ++aa) {
            P[q++] = __fmul_rn(S[aa].x, S[bb].x);
            P[q++] = __fmul_rn(S[aa].y, S[bb].y);
            P[q++] = __fmul_rn(S[aa].z, S[bb].z);
          }
      } else {
        // pairs in the order (0,1) (0,2) (1,2) (0,3) (1,3) (2,3)
        int q = 0;
#pragma unroll
        for (int bb = 1; bb < NR; ++bb)
#pragma unroll
          for (int aa = 0; aa < bb; ++aa) P[q++] = dot3(S[aa], S[bb]);
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        a0[q] = __fadd_rn(a0[q], P[q]);
#pragma unroll
        for (int d = 0; d < 3; ++d) ak[q][d] = fma2(f2(P[q]), tk[d], ak[q][d]);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[b]);
    if (warp == 0 && k + MS_STAGES < n_sub) {
      if (!__all_sync(0xffffffffu, mbar_wait(&empty[b], ph, p.timeout_ns))) {
        ok = false;
        break;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(k + MS_STAGES);
      issued = k + MS_STAGES + 1;
    }
  }
  if (!ok) {
    // a wait ran out: flag it and give the copies this block issued a
    // bounded time to land; the block's partials are not used
    if (lane == 0) atomicExch(p.err, 1u);
    if (warp == 0)
      for (int q = k; q < issued; ++q)
        mbar_wait(&full[q % MS_STAGES], (uint32_t)(q / MS_STAGES) & 1u, p.timeout_ns);
  }

  // site groups of a warp share slots: add them (fixed butterfly order)
  for (int o = TL; o < 32; o <<= 1) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      a0[q] += __shfl_xor_sync(0xffffffffu, a0[q], o);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        ak[q][d].x += __shfl_xor_sync(0xffffffffu, ak[q][d].x, o);
        ak[q][d].y += __shfl_xor_sync(0xffffffffu, ak[q][d].y, o);
      }
    }
  }
  // warps in order, FP32 (GB300's FP64 rate is a small fraction of its FP32
  // rate); the block's sums leave as FP64
  for (int w = 0; w < NW; ++w) {
    if (warp == w && grp == 0 && live) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        float* rv = &red[q * NM][lane];
        const float v[NM] = {a0[q], ak[q][0].x, ak[q][0].y, ak[q][1].x, ak[q][1].y, ak[q][2].x, ak[q][2].y};
#pragma unroll
        for (int m = 0; m < NM; ++m) rv[m * 32] = (w == 0 ? 0.0f : rv[m * 32]) + v[m];
      }
    }
    __syncthreads();
  }
  double* out = p.partials + (((long long)s * p.n_tiles + blockIdx.x) * R_T + 32 * round) * NV;
  for (int i = threadIdx.x; i < nt * NV; i += MEAS_BS) out[i] = (double)red[i % NV][i / NV];
}

// One warp per (sample, slot, value): lane l adds the partials of blocks
// l, l + 32, ... in that order, then the lanes are added in a fixed butterfly;
// the total times 1/N.  Eight values per block of 256 threads.
template <int MODE>
__global__ void __launch_bounds__(256) k_meas_final_staged(const OverlapParams p, int NV) {
  const int t = blockIdx.x % p.R_T, s = blockIdx.x / p.R_T;
  const int v = blockIdx.y * 8 + (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (v >= NV) return;
  const SampleDev& sd = p.samples[s];
  const int n_tiles = (int)(((long long)sd.N + p.tile_ss - 1) / p.tile_ss);
  const long long stride = (long long)p.R_T * NV;
  const double* src = p.partials + ((long long)s * p.n_tiles * p.R_T + t) * NV + v;
  double acc = 0.0;
#pragma unroll 4
  for (int k = lane; k < n_tiles; k += 32) acc += src[k * stride];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane != 0) return;
  const double val = acc / (double)sd.N;
  const int q = v / NM, m = v % NM;
  if constexpr (MODE == MEAS_QTENSOR) {
    if (m == 0) {
      if (p.D) p.D[((long long)s * p.R_T + t) * 9 + q] = val;
    } else if (p.C) {
      const int d = (m - 1) / 2, ri = (m - 1) % 2;
      p.C[(((long long)s * p.R_T + t) * 3 + d) * 18 + q * 2 + ri] = val;
    }
  } else if constexpr (MODE == MEAS_CHIRAL) {
    if (p.C) {
      const int mode = m == 0 ? 0 : 1 + (m - 1) / 2, ri = m == 0 ? 0 : (m - 1) % 2;
      double* dst = p.C + (((long long)s * p.R_T + t) * p.n_pairs + q / 3) * 24 + (q % 3) * 8;
      dst[2 * mode + ri] = val;
      if (m == 0) dst[1] = 0.0;
    }
  } else if (p.D) {
    const int mode = m == 0 ? 0 : 1 + (m - 1) / 2, ri = m == 0 ? 0 : (m - 1) % 2;
    double* dst = p.D + (((long long)s * p.R_T + t) * p.n_pairs + q) * 8;
    dst[2 * mode + ri] = val;
    if (m == 0) dst[1] = 0.0;
  }
}

template <int F, int MODE, int NR>
static cudaError_t staged_launch(const OverlapParams& p, cudaStream_t st) {
  constexpr int NV = staged_products<MODE, NR>() * NM;
  const int smem = MS_STAGES * FmtInfo<F>::PLANES * p.Gu * p.grow;
  cudaError_t e = cudaFuncSetAttribute(k_meas_staged<F, MODE, NR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid(p.n_tiles, (p.R_T + 31) / 32, p.n_samples);
  k_meas_staged<F, MODE, NR><<<grid, MEAS_BS, smem, st>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_meas_final_staged<MODE><<<dim3(p.n_samples * p.R_T, (NV + 7) / 8), 256, 0, st>>>(p, NV);
  return cudaGetLastError();
}

template <int F, int MODE>
static cudaError_t meas_launch(const OverlapParams& p, cudaStream_t st) {
  const dim3 grid(p.n_tiles * p.n_pairs, p.n_samples);
  k_meas_tiles<F, MODE><<<grid, MEAS_BS, 0, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  constexpr int NVAL = n_products<MODE>() * NM;
  k_meas_final<MODE><<<dim3(p.n_samples * p.n_pairs * p.R_T, (NVAL + 7) / 8), 256, 0, st>>>(p);
  return cudaGetLastError();
}

template <int F>
static cudaError_t meas_fmt(const OverlapParams& p, int mode, cudaStream_t st) {
  if (p.sub > 0 && mode == MEAS_QTENSOR) return staged_launch<F, MEAS_QTENSOR, 2>(p, st);
  if (p.sub > 0 && mode == MEAS_PAIRS) {
    switch (min(p.R_O, 4)) {
      case 2: return staged_launch<F, MEAS_PAIRS, 2>(p, st);
      case 3: return staged_launch<F, MEAS_PAIRS, 3>(p, st);
      case 4: return staged_launch<F, MEAS_PAIRS, 4>(p, st);
    }
    return cudaErrorInvalidValue;
  }
  switch (mode) {
    case MEAS_QTENSOR: return meas_launch<F, MEAS_QTENSOR>(p, st);
    case MEAS_PAIRS: return meas_launch<F, MEAS_PAIRS>(p, st);
    case MEAS_PAIRS_CHIRAL: return meas_launch<F, MEAS_PAIRS_CHIRAL>(p, st);
  }
  return cudaErrorInvalidValue;
}

static cudaError_t meas_dispatch(int fmt, const OverlapParams& p, int mode, cudaStream_t st) {
  switch (fmt) {
    case FMT_F32: return meas_fmt<FMT_F32>(p, mode, st);
    case FMT_F16: return meas_fmt<FMT_F16>(p, mode, st);
    case FMT_BF16: return meas_fmt<FMT_BF16>(p, mode, st);
    case FMT_ANG16: return meas_fmt<FMT_ANG16>(p, mode, st);
    case FMT_OCT16: return meas_fmt<FMT_OCT16>(p, mode, st);
    case FMT_YX4: return meas_fmt<FMT_YX4>(p, mode, st);
  }
  return cudaErrorInvalidValue;
}

// Local chirality of every site for the chunk groups g < Gu (Sec. 2):
// kappa_i^a = s_{i+a} . (s_i x s_{i-a}) along a = x, y, z, written as binary32
// in the chunk layout of the spins ([a][g][ss][4 systems]), so that the staged
// kernel forms the chiral pair overlaps from it as it forms D from spins.  One
// launch per parity over the sweep block table; a thread owns one site and
// walks its chunk groups, as the sweeps do.
template <int F>
__global__ void __launch_bounds__(SWEEP_BS) k_chirality(const ChiralityParams p) {
  constexpr int VEC = 4, PL = FmtInfo<F>::PLANES;
  using Chunk = typename FmtInfo<F>::Chunk;
  const int4 blk = p.blocks[blockIdx.x];
  const SampleDev& sd = p.samples[blk.x];
  const uint32_t h = (uint32_t)blk.z + threadIdx.x;
  if (h >= ((uint32_t)sd.N >> 1)) return;
  const int g0 = blk.y * p.GPT, g1 = min(p.Gu, min(p.G, g0 + p.GPT));
  if (g0 >= g1) return;
  const SiteGeom gm = site_geom(sd, h, p.parity);        // neighbours +x, -x, +y, -y, +z, -z
  const unsigned char* base = p.spins + sd.spin_off;
  const long long ps = sd.plane_stride;
  const SampleDev& kd = p.ksamples[blk.x];
  unsigned char* kb = p.kappa + kd.spin_off;
  const long long kps = kd.plane_stride;
  for (int g = g0; g < g1; ++g) {
    Chunk c[PL];
    load_chunks<F, LD_RO>(base + chunk_offset<F>(sd, g, gm.own), ps, c);
    Spins<VEC> s0;
    decode<F>(c, s0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Chunk cp[PL], cm[PL];
      load_chunks<F, LD_RO>(base + chunk_offset<F>(sd, g, gm.nb[2 * a]), ps, cp);
      load_chunks<F, LD_RO>(base + chunk_offset<F>(sd, g, gm.nb[2 * a + 1]), ps, cm);
      Spins<VEC> sp, sm;
      decode<F>(cp, sp);
      decode<F>(cm, sm);
      float k4[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        const int q = v >> 1;
        const bool hi = v & 1;
        const V3 A = {hi ? sp.x[q].y : sp.x[q].x, hi ? sp.y[q].y : sp.y[q].x, hi ? sp.z[q].y : sp.z[q].x};
        const V3 Bv = {hi ? s0.x[q].y : s0.x[q].x, hi ? s0.y[q].y : s0.y[q].x, hi ? s0.z[q].y : s0.z[q].x};
        const V3 Cv = {hi ? sm.x[q].y : sm.x[q].x, hi ? sm.y[q].y : sm.y[q].x, hi ? sm.z[q].y : sm.z[q].x};
        k4[v] = triple(A, Bv, Cv);
      }
      *reinterpret_cast<float4*>(kb + a * kps + ((long long)g * sd.N + gm.own) * 16) =
          make_float4(k4[0], k4[1], k4[2], k4[3]);
    }
  }
}

cudaError_t launch_chirality(int fmt, const ChiralityParams& p, int n_blocks, cudaStream_t st) {
  switch (fmt) {
    case FMT_F32: k_chirality<FMT_F32><<<n_blocks, SWEEP_BS, 0, st>>>(p); break;
    case FMT_F16: k_chirality<FMT_F16><<<n_blocks, SWEEP_BS, 0, st>>>(p); break;
    case FMT_BF16: k_chirality<FMT_BF16><<<n_blocks, SWEEP_BS, 0, st>>>(p); break;
    case FMT_ANG16: k_chirality<FMT_ANG16><<<n_blocks, SWEEP_BS, 0, st>>>(p); break;
    case FMT_OCT16: k_chirality<FMT_OCT16><<<n_blocks, SWEEP_BS, 0, st>>>(p); break;
    case FMT_YX4: k_chirality<FMT_YX4><<<n_blocks, SWEEP_BS, 0, st>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// chiral pair overlaps from the binary32 chirality buffer (staged kernel)
cudaError_t launch_chiral_staged(const OverlapParams& p, cudaStream_t st) {
  switch (min(p.R_O, 4)) {
    case 2: return staged_launch<FMT_F32, MEAS_CHIRAL, 2>(p, st);
    case 3: return staged_launch<FMT_F32, MEAS_CHIRAL, 3>(p, st);
    case 4: return staged_launch<FMT_F32, MEAS_CHIRAL, 4>(p, st);
  }
  return cudaErrorInvalidValue;
}

int meas_partial_values(bool qtensor, bool chiral) {
  return (qtensor ? 3 : (chiral ? 4 : 1)) * NM;
}

StagedGeom staged_geometry(int fmt, bool qtensor, int R_O, int R_T, long long n_max,
                           long long n_total) {
  StagedGeom g{};
  int planes = 3, chunk = 8;
  switch (fmt) {
    case FMT_F32: planes = FmtInfo<FMT_F32>::PLANES; chunk = FmtInfo<FMT_F32>::CHUNK; break;
    case FMT_F16: planes = FmtInfo<FMT_F16>::PLANES; chunk = FmtInfo<FMT_F16>::CHUNK; break;
    case FMT_BF16: planes = FmtInfo<FMT_BF16>::PLANES; chunk = FmtInfo<FMT_BF16>::CHUNK; break;
    case FMT_ANG16: planes = FmtInfo<FMT_ANG16>::PLANES; chunk = FmtInfo<FMT_ANG16>::CHUNK; break;
    case FMT_OCT16: planes = FmtInfo<FMT_OCT16>::PLANES; chunk = FmtInfo<FMT_OCT16>::CHUNK; break;
    case FMT_YX4: planes = FmtInfo<FMT_YX4>::PLANES; chunk = FmtInfo<FMT_YX4>::CHUNK; break;
    default: return g;
  }
  const int r_use = qtensor ? 2 : std::min(R_O, 4);
  if (r_use < 2) return g;
  g.Gu = (r_use * R_T + 3) / 4;               // chunk groups of memory slots [0, r_use R_T)
  g.values = (qtensor ? 9 : r_use * (r_use - 1) / 2) * NM;
  // rows padded by 16 bytes put consecutive chunk groups 4 banks apart
  constexpr long long budget = 96 * 1024;
  for (int sub = 64; sub >= 8 && !g.ok; sub >>= 1) {
    const int grow = sub * chunk + 16;
    const long long bytes = (long long)MS_STAGES * planes * g.Gu * grow;
    if (bytes <= budget) {
      g.ok = 1;
      g.sub = sub;
      g.grow = grow;
      g.smem = (int)bytes;
    }
  }
  if (!g.ok) return g;
  g.rounds = (R_T + 31) / 32;
  // about 8 blocks per SM over the whole call; a lane's FP32 sums stay short
  long long per = (n_total * g.rounds + 1215) / 1216;
  per = (per + g.sub - 1) / g.sub * g.sub;
  g.tile_ss = (int)std::min<long long>(8192, std::max<long long>(g.sub, per));
  g.n_tiles = (int)((n_max + g.tile_ss - 1) / g.tile_ss);
  return g;
}

cudaError_t launch_overlaps(int fmt, const OverlapParams& p, bool chiral, cudaStream_t st) {
  return meas_dispatch(fmt, p, chiral ? MEAS_PAIRS_CHIRAL : MEAS_PAIRS, st);
}

cudaError_t launch_qtensor(int fmt, const OverlapParams& p, cudaStream_t st) {
  return meas_dispatch(fmt, p, MEAS_QTENSOR, st);
}

}  // namespace hsg
