// Multi-hit tile updates: the paper's double checkerboard (Sec. 3.2; Table 1,
// "10 x (1 HB + 10 OR)").  The lattice is cut into cubic tiles of edge T,
// coloured by the parity of their tile coordinates; L / T is even, so no two
// tiles of one colour share a bond.  One launch updates every tile of one
// colour: a block owns one tile and one chunk group (4 systems), reads the
// tile and its face halo once into shared memory (as stored for 16-bit
// components, decoded to FP32 otherwise), runs
// n_rounds x (n_or over-relaxation + n_hb heat-bath) tile sweeps there, each
// the tile's even sites and then its odd sites, with the halo fixed, and
// writes the tile back.  The k-th tile sweep of a launch keys its heat-bath
// numbers with the sample's sweep counter + k, as a lattice sweep does.
//
// Every update goes through the storage codec (encode, decode) before it is
// written to shared memory, so the tile holds exactly what storage would
// hold after each sweep, and the thread writes back the chunk it encoded
// last.  The arithmetic is that of the lattice sweeps (field in the order
// +x, -x, +y, -y, +z, -z, then the field H; the same moves), so a tile sweep
// computes what a lattice sweep restricted to the tile computes.
#include "hsg_kernels.cuh"

namespace hsg {

namespace {

// Shared-memory layout of a tile (edge T) and its face halo, per parity and
// component: "main" holds the sites with x in [0, T) of the padded rows
// (y, z in [-1, T]), T/2 per row and parity, so the four threads of a row and
// the next row read eight consecutive entries (no bank conflict); "xhalo"
// holds, per interior row and parity, the one halo site of that parity
// (x = -1 or x = T).  Both sit in one array with one component stride.
template <int T>
struct TileShape {
  static constexpr int P = T + 2;                 // padded rows per plane, planes
  static constexpr int NM = P * P * (T / 2);      // main entries of one parity
  static constexpr int NR = P * P;                // xhalo entries (one per padded row)
  static constexpr int CS = NM + NR;              // component stride
  static constexpr int NT = T * T * T / 2;        // threads: the tile's sites of one parity
};

template <int T>
__device__ __forceinline__ int row_of(int y, int z) { return (z + 1) * (T + 2) + (y + 1); }

// entry of padded local (x, y, z) in the array of its parity
template <int T>
__device__ __forceinline__ int tentry(int x, int y, int z) {
  return (x < 0 || x >= T) ? TileShape<T>::NM + row_of<T>(y, z) : row_of<T>(y, z) * (T / 2) + (x >> 1);
}

// What shared memory holds per (site, component): the four systems' binary16
// or bfloat16 values as stored, or the decoded binary32 values (formats whose
// decode is not a conversion).
template <int F> struct Sh { using E = float4; static constexpr bool RAW = false; };
template <> struct Sh<FMT_F16> { using E = uint2; static constexpr bool RAW = true; };
template <> struct Sh<FMT_BF16> { using E = uint2; static constexpr bool RAW = true; };

template <int F>
__device__ __forceinline__ float2 raw2f(uint32_t w) {
  if constexpr (F == FMT_F16) return h2f(w);
  else return b2f(w);
}

template <int F>
__device__ __forceinline__ void sh_read(const typename Sh<F>::E* A, int cs, int q, Spins<4>& v) {
  if constexpr (Sh<F>::RAW) {
    const uint2 a = A[q], b = A[cs + q], c = A[2 * cs + q];
    v.x[0] = raw2f<F>(a.x);
    v.x[1] = raw2f<F>(a.y);
    v.y[0] = raw2f<F>(b.x);
    v.y[1] = raw2f<F>(b.y);
    v.z[0] = raw2f<F>(c.x);
    v.z[1] = raw2f<F>(c.y);
  } else {
    const float4 a = A[q], b = A[cs + q], c = A[2 * cs + q];
    v.x[0] = make_float2(a.x, a.y);
    v.x[1] = make_float2(a.z, a.w);
    v.y[0] = make_float2(b.x, b.y);
    v.y[1] = make_float2(b.z, b.w);
    v.z[0] = make_float2(c.x, c.y);
    v.z[1] = make_float2(c.z, c.w);
  }
}

// store an encoded chunk (RAW) or its decoded values
template <int F>
__device__ __forceinline__ void sh_write(typename Sh<F>::E* A, int cs, int q,
                                         const typename FmtInfo<F>::Chunk* c) {
  if constexpr (Sh<F>::RAW) {
    A[q] = c[0];
    A[cs + q] = c[1];
    A[2 * cs + q] = c[2];
  } else {
    Spins<4> v;
    decode<F>(c, v);
    A[q] = make_float4(v.x[0].x, v.x[0].y, v.x[1].x, v.x[1].y);
    A[cs + q] = make_float4(v.y[0].x, v.y[0].y, v.y[1].x, v.y[1].y);
    A[2 * cs + q] = make_float4(v.z[0].x, v.z[0].y, v.z[1].x, v.z[1].y);
  }
}

}  // namespace

// Binary32 tiles: at most 80 registers per thread, i.e. 3 blocks of 256 threads
// (T = 8) or 24 of 32 (T = 4) per SM; unbounded they take 92-99 registers and
// run 2 blocks per SM.  The 16-bit formats compile to 80 registers unbounded.
template <int F, int T>
constexpr int multihit_min_blocks() { return F == FMT_F32 ? (T == 8 ? 3 : 24) : 0; }

template <int F, bool J16, bool FAST, int T>
__global__ void __launch_bounds__(TileShape<T>::NT, multihit_min_blocks<F, T>()) k_multihit(const MultihitParams p) {
  using TS = TileShape<T>;
  using E = typename Sh<F>::E;
  constexpr int VEC = 4, PL = FmtInfo<F>::PLANES;
  constexpr bool MIXED = (F == FMT_F16) && J16;     // f16 x f16 products, exact in f32
  using Chunk = typename FmtInfo<F>::Chunk;
  __shared__ E A[2][3 * TS::CS];                    // [parity][component][entry]
  const int4 blk = p.blocks[p.blk_base + (int)blockIdx.x];     // (sample, tile, chunk group)
  if (!p.active[blk.x]) return;                               // the whole block: one sample
  const SampleDev sd = p.samples[blk.x];
  const int L = sd.L, B = L / T, g = blk.z;
  const int X0 = (blk.y % B) * T, Y0 = ((blk.y / B) % B) * T, Z0 = (blk.y / (B * B)) * T;
  unsigned char* base = p.spins + sd.spin_off;
  const long long ps = sd.plane_stride;
  const uint32_t half_n = (uint32_t)sd.N >> 1;
  // storage site and natural site index of padded local (x, y, z); the tile's
  // origin is even and L is even, so local and global parities agree
  auto locate = [&](int x, int y, int z, uint32_t& site) -> uint32_t {
    const int gx = X0 + x < 0 ? L - 1 : (X0 + x >= L ? 0 : X0 + x);
    const int gy = Y0 + y < 0 ? L - 1 : (Y0 + y >= L ? 0 : Y0 + y);
    const int gz = Z0 + z < 0 ? L - 1 : (Z0 + z >= L ? 0 : Z0 + z);
    site = (uint32_t)gx + (uint32_t)L * ((uint32_t)gy + (uint32_t)L * (uint32_t)gz);
    return (uint32_t)((gx + gy + gz) & 1) * half_n + (site >> 1);
  };
  auto fetch = [&](int x, int y, int z) {
    uint32_t site;
    const uint32_t ss = locate(x, y, z, site);
    Chunk c[PL];
    load_chunks<F, LD_RO>(base + chunk_offset<F>(sd, g, ss), ps, c);
    sh_write<F>(A[(x + y + z) & 1], TS::CS, tentry<T>(x, y, z), c);
  };

  // the tile and its face halo (edges and corners are no site's neighbours):
  // main entries of padded rows with y or z inside, then the x-halo sites
  for (int i = threadIdx.x; i < 2 * TS::NM; i += TS::NT) {
    const int par = i / TS::NM, e = i - par * TS::NM;
    const int xh = e % (T / 2), row = e / (T / 2);
    const int y = row % TS::P - 1, z = row / TS::P - 1;
    if ((y < 0 || y >= T) && (z < 0 || z >= T)) continue;
    fetch(2 * xh + ((par + y + z) & 1), y, z);
  }
  for (int i = threadIdx.x; i < 2 * T * T; i += TS::NT) {
    const int par = i / (T * T), e = i - par * T * T;
    const int y = e % T, z = e / T;
    fetch(((y + z + 1) & 1) == par ? -1 : T, y, z);
  }

  // this thread's two sites, one of each parity
  const int t = threadIdx.x;
  const int xh = t % (T / 2), y = (t / (T / 2)) % T, z = t / ((T / 2) * T);
  int own[2], nb[2][6];
  uint32_t gsite[2], gss[2];
  float j6[2][6], h3[2][3];
  uint32_t jh[2][6];
#pragma unroll
  for (int par = 0; par < 2; ++par) {
    const int x = 2 * xh + ((par + y + z) & 1);
    own[par] = tentry<T>(x, y, z);
    nb[par][0] = tentry<T>(x + 1, y, z);
    nb[par][1] = tentry<T>(x - 1, y, z);
    nb[par][2] = tentry<T>(x, y + 1, z);
    nb[par][3] = tentry<T>(x, y - 1, z);
    nb[par][4] = tentry<T>(x, y, z + 1);
    nb[par][5] = tentry<T>(x, y, z - 1);
    gss[par] = locate(x, y, z, gsite[par]);
    load_record<J16>(p.rec, sd.rec_off + gss[par], j6[par], h3[par]);
    if (MIXED) load_record_j16(p.rec, sd.rec_off + gss[par], jh[par]);
  }
  const uint32_t sys0 = (uint32_t)sd.sys_base + (uint32_t)g * VEC;   // even
  float bt[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) bt[v] = p.beta[(long long)blk.x * p.Wp + g * VEC + v];
  const uint32_t sweep0 = (uint32_t)p.counters[2 * blk.x];
  __syncthreads();

  Chunk keep[2][PL];            // the last encoded state of the thread's two sites
  const int per = p.n_or + p.n_hb;
  for (int r = 0; r < p.n_rounds; ++r) {
    for (int k = 0; k < per; ++k) {
      const bool hb = k >= p.n_or;
      const uint32_t sweep = sweep0 + (uint32_t)(r * per + k);
#pragma unroll
      for (int par = 0; par < 2; ++par) {
        const E* O = A[par ^ 1];
        // local field h = sum_n J_n s_n + H, in the order +x, -x, +y, -y, +z, -z
        Spins<VEC> hf;
        if constexpr (MIXED) {
#pragma unroll
          for (int q = 0; q < VEC / 2; ++q) {
            hf.x[q] = make_float2(0.0f, 0.0f);
            hf.y[q] = make_float2(0.0f, 0.0f);
            hf.z[q] = make_float2(0.0f, 0.0f);
          }
#pragma unroll
          for (int n = 0; n < 6; ++n) {
            const uint2 a = O[nb[par][n]], b = O[TS::CS + nb[par][n]], c = O[2 * TS::CS + nb[par][n]];
            fma_f16_pair(hf.x[0], a.x, jh[par][n]);
            fma_f16_pair(hf.x[1], a.y, jh[par][n]);
            fma_f16_pair(hf.y[0], b.x, jh[par][n]);
            fma_f16_pair(hf.y[1], b.y, jh[par][n]);
            fma_f16_pair(hf.z[0], c.x, jh[par][n]);
            fma_f16_pair(hf.z[1], c.y, jh[par][n]);
          }
        } else {
          {
            Spins<VEC> nbv;
            sh_read<F>(O, TS::CS, nb[par][0], nbv);
            const float2 jj = f2(j6[par][0]);
#pragma unroll
            for (int q = 0; q < VEC / 2; ++q) {
              hf.x[q] = mul2(jj, nbv.x[q]);
              hf.y[q] = mul2(jj, nbv.y[q]);
              hf.z[q] = mul2(jj, nbv.z[q]);
            }
          }
#pragma unroll
          for (int n = 1; n < 6; ++n) {
            Spins<VEC> nbv;
            sh_read<F>(O, TS::CS, nb[par][n], nbv);
            const float2 jj = f2(j6[par][n]);
#pragma unroll
            for (int q = 0; q < VEC / 2; ++q) {
              hf.x[q] = fma2(jj, nbv.x[q], hf.x[q]);
              hf.y[q] = fma2(jj, nbv.y[q], hf.y[q]);
              hf.z[q] = fma2(jj, nbv.z[q], hf.z[q]);
            }
          }
        }
        {
          const float2 hx = f2(h3[par][0]), hy = f2(h3[par][1]), hz = f2(h3[par][2]);
#pragma unroll
          for (int q = 0; q < VEC / 2; ++q) {
            hf.x[q] = add2(hf.x[q], hx);
            hf.y[q] = add2(hf.y[q], hy);
            hf.z[q] = add2(hf.z[q], hz);
          }
        }
        Spins<VEC> s;
        sh_read<F>(A[par], TS::CS, own[par], s);
        if (hb) {
#pragma unroll
          for (int q = 0; q < VEC / 2; ++q) {
            const uint4 rn =
                philox4x32_10_rk(make_uint4(gsite[par], (sys0 >> 1) + q, sweep, TAG_HB), p.rk);
            hb_move<FAST>(s.x[q].x, s.y[q].x, s.z[q].x, hf.x[q].x, hf.y[q].x, hf.z[q].x,
                          bt[2 * q], u01(rn.x), u01(rn.y));
            hb_move<FAST>(s.x[q].y, s.y[q].y, s.z[q].y, hf.x[q].y, hf.y[q].y, hf.z[q].y,
                          bt[2 * q + 1], u01(rn.z), u01(rn.w));
          }
        } else {
#pragma unroll
          for (int q = 0; q < VEC / 2; ++q) or_move2(s.x[q], s.y[q], s.z[q], hf.x[q], hf.y[q], hf.z[q]);
        }
        // through the storage codec, as a stored spin would be
        encode<F>(s, keep[par]);
        sh_write<F>(A[par], TS::CS, own[par], keep[par]);
        __syncthreads();
      }
    }
  }
#pragma unroll
  for (int par = 0; par < 2; ++par) store_chunks<F>(base + chunk_offset<F>(sd, g, gss[par]), ps, keep[par]);
}

template <int F, bool J16, bool FAST>
static cudaError_t mh_tile(int tile, const MultihitParams& p, int n_blocks, cudaStream_t st) {
  if (tile == 4) {
    k_multihit<F, J16, FAST, 4><<<n_blocks, TileShape<4>::NT, 0, st>>>(p);
  } else if (tile == 8) {
    k_multihit<F, J16, FAST, 8><<<n_blocks, TileShape<8>::NT, 0, st>>>(p);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int F>
static cudaError_t mh_fmt(bool j16, bool fast, int tile, const MultihitParams& p, int n_blocks,
                          cudaStream_t st) {
  if (j16) return fast ? mh_tile<F, true, true>(tile, p, n_blocks, st) : mh_tile<F, true, false>(tile, p, n_blocks, st);
  return fast ? mh_tile<F, false, true>(tile, p, n_blocks, st) : mh_tile<F, false, false>(tile, p, n_blocks, st);
}

cudaError_t launch_multihit(int fmt, bool j16, bool fast, int tile, const MultihitParams& p,
                            int n_blocks, cudaStream_t st) {
  if (n_blocks <= 0) return cudaSuccess;
  switch (fmt) {
    case FMT_F32: return mh_fmt<FMT_F32>(j16, fast, tile, p, n_blocks, st);
    case FMT_F16: return mh_fmt<FMT_F16>(j16, fast, tile, p, n_blocks, st);
    case FMT_BF16: return mh_fmt<FMT_BF16>(j16, fast, tile, p, n_blocks, st);
    case FMT_ANG16: return mh_fmt<FMT_ANG16>(j16, fast, tile, p, n_blocks, st);
    case FMT_OCT16: return mh_fmt<FMT_OCT16>(j16, fast, tile, p, n_blocks, st);
    case FMT_YX4: return mh_fmt<FMT_YX4>(j16, fast, tile, p, n_blocks, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hsg
