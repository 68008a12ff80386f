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
// tile order.  (GB300's FP64 rate is a small fraction of its FP32 rate, so FP64
// work is kept per tile, not per site.)
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
enum { MEAS_QTENSOR = 0, MEAS_PAIRS = 1, MEAS_PAIRS_CHIRAL = 2 };

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

// One block per (sample, unit, slot): value v of the slot is the sum of the
// tiles' partials in tile order (4 threads per value, each a contiguous range
// of tiles, then added in range order), times 1/N.
template <int MODE>
__global__ void __launch_bounds__(256) k_meas_final(const OverlapParams p) {
  constexpr int NP = n_products<MODE>();
  constexpr int NVAL = NP * NM;
  const int t = blockIdx.x % p.R_T, su = blockIdx.x / p.R_T;
  const int unit = su % p.n_pairs, s = su / p.n_pairs;
  const SampleDev& sd = p.samples[s];
  const int n_tiles = (int)(((long long)sd.N + MEAS_TILE - 1) / MEAS_TILE);
  __shared__ double part[4][64];
  const int v = threadIdx.x % 64, q4 = threadIdx.x / 64;
  double acc = 0.0;
  if (v < NVAL) {
    const int per = (n_tiles + 3) / 4;
    const double* src = p.partials + ((long long)s * p.n_pairs + unit) * p.n_tiles * p.R_T * NVAL +
                        (long long)t * NVAL + v;
    for (int k = q4 * per; k < min(n_tiles, (q4 + 1) * per); ++k) acc += src[(long long)k * p.R_T * NVAL];
  }
  part[q4][v] = acc;
  __syncthreads();
  if (threadIdx.x >= NVAL) return;
  const double sum = ((part[0][v] + part[1][v]) + part[2][v]) + part[3][v];
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

template <int F, int MODE>
static cudaError_t meas_launch(const OverlapParams& p, cudaStream_t st) {
  const dim3 grid(p.n_tiles * p.n_pairs, p.n_samples);
  k_meas_tiles<F, MODE><<<grid, MEAS_BS, 0, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_meas_final<MODE><<<p.n_samples * p.n_pairs * p.R_T, 256, 0, st>>>(p);
  return cudaGetLastError();
}

template <int F>
static cudaError_t meas_fmt(const OverlapParams& p, int mode, cudaStream_t st) {
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

int meas_partial_values(bool qtensor, bool chiral) {
  return (qtensor ? 3 : (chiral ? 4 : 1)) * NM;
}

cudaError_t launch_overlaps(int fmt, const OverlapParams& p, bool chiral, cudaStream_t st) {
  return meas_dispatch(fmt, p, chiral ? MEAS_PAIRS_CHIRAL : MEAS_PAIRS, st);
}

cudaError_t launch_qtensor(int fmt, const OverlapParams& p, cudaStream_t st) {
  return meas_dispatch(fmt, p, MEAS_QTENSOR, st);
}

}  // namespace hsg
