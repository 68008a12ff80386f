/*
 * FP64 CPU oracle for the checkerboard heat-bath / over-relaxation / parallel
 * tempering Monte Carlo of the 3D Edwards-Anderson Heisenberg spin glass in a
 * random field (Yavors'kii & Weigel, arXiv:1204.6192).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the CUDA library.  Plain loops in the
 * order of the paper's definitions, every floating-point value in binary64,
 * built with -ffp-contract=off so that no multiply-add is fused.
 *
 * Readings of the paper fixed here (the paper leaves them open):
 *  - Eq. (1) counts each nearest-neighbour bond once, so that the local field
 *    H_eff = sum_j J_ij s_j + H_i of Eq. (2) is minus the gradient of E.
 *  - The heat-bath draw of Eq. (2) is not printed in the paper (it points to
 *    Lee & Young); it is the inverse CDF of the density exp(a cos t) on
 *    cos t in [-1, 1], written with log1p/expm1, plus a uniform azimuth around
 *    the field in the Duff et al. (JCGT 2017) orthonormal frame.
 *  - Every move is followed by s <- s / |s| (then the storage codec, if any).
 *  - Parallel tempering (Eq. 4) walks the pairs (k, k+1) upwards from the
 *    lowest temperature and swaps temperatures, not spins.
 */
#include "hsg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3" (SC'11): 10 rounds of two 32x32->64 multiplications with */
/* the round multipliers, xor with the other half and the key, key bumped by */
/* the two Weyl constants between rounds.                                    */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_MUL_A = 0xD2511F53u;
static const uint32_t PHILOX_MUL_B = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL_A = 0x9E3779B9u;
static const uint32_t PHILOX_WEYL_B = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_MUL_A * (uint64_t)x0;
    uint64_t p1 = (uint64_t)PHILOX_MUL_B * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += PHILOX_WEYL_A;
    k1 += PHILOX_WEYL_B;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_philox_many(const uint32_t* ctr, long n, uint64_t seed, uint32_t* out) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (long k = 0; k < n; ++k) orc_philox4x32_10(ctr + 4 * k, key, out + 4 * k);
}

/* u = (2*(x >> 9) + 1) / 2^24: 2^23 equally spaced points strictly inside (0,1) */
double orc_uniform(uint32_t x) {
  return (double)(2u * (x >> 9) + 1u) * (1.0 / 16777216.0);
}

/* the pair of uniforms a system draws from one Philox block (two systems share one) */
static void pair_uniforms(uint32_t c0, uint64_t gsys, uint32_t c2, uint32_t tag,
                          uint64_t seed, double* u1, double* u2) {
  uint32_t ctr[4] = {c0, (uint32_t)(gsys >> 1), c2, tag};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  int b = (int)(gsys & 1u);
  *u1 = orc_uniform(out[2 * b]);
  *u2 = orc_uniform(out[2 * b + 1]);
}

/* ------------------------------------------------------------------------ */
/* Storage codecs: what a spin becomes after it is stored and read back.     */
/* ------------------------------------------------------------------------ */

/* nearest value with a p-bit significand (p counts the hidden bit), ties to even,
   for |x| >= 2^emin; below that the spacing is fixed at 2^(emin - p + 1) */
static double round_to_format(double x, int p, int emin) {
  if (x == 0.0 || !isfinite(x)) return x;
  int e;
  frexp(fabs(x), &e);            /* |x| = m * 2^e, m in [0.5, 1) */
  int exp2 = e - 1;              /* |x| in [2^exp2, 2^(exp2+1)) */
  if (exp2 < emin) exp2 = emin;
  double ulp = ldexp(1.0, exp2 - (p - 1));
  return nearbyint(x / ulp) * ulp;   /* default rounding mode: ties to even */
}

double orc_round_fp16(double x) { return round_to_format(x, 11, -14); }
double orc_round_bf16(double x) { return round_to_format(x, 8, -126); }

static double sgn_nonneg(double v) { return v >= 0.0 ? 1.0 : -1.0; }

void orc_codec_roundtrip(double v[3], int codec) {
  switch (codec) {
    case ORC_CODEC_NONE:
      return;
    case ORC_CODEC_FP16:
      for (int c = 0; c < 3; ++c) v[c] = orc_round_fp16(v[c]);
      return;
    case ORC_CODEC_BF16:
      for (int c = 0; c < 3; ++c) v[c] = orc_round_bf16(v[c]);
      return;
    case ORC_CODEC_FP32:
      /* binary32 storage: nearest float, ties to even (C's double -> float conversion) */
      for (int c = 0; c < 3; ++c) v[c] = (double)(float)v[c];
      return;
    case ORC_CODEC_ANGLE16: {
      /* polar angle theta in [0, pi] on 65536 levels, azimuth on a 2^16 ring */
      double z = v[2];
      if (z > 1.0) z = 1.0;
      if (z < -1.0) z = -1.0;
      double theta = acos(z);
      double phi = atan2(v[1], v[0]);
      long tq = (long)floor(theta / ORC_PI * 65535.0 + 0.5);
      if (tq > 65535) tq = 65535;
      long pq = ((long)floor(phi / (2.0 * ORC_PI) * 65536.0 + 0.5)) & 0xffff;
      double th = (double)tq * ORC_PI / 65535.0;
      double ph = (double)pq * 2.0 * ORC_PI / 65536.0;
      v[0] = sin(th) * cos(ph);
      v[1] = sin(th) * sin(ph);
      v[2] = cos(th);
      return;
    }
    case ORC_CODEC_OCT16: {
      /* octahedral map (Cigolle et al., JCGT 2014) on a 16-bit signed grid */
      double l1 = fabs(v[0]) + fabs(v[1]) + fabs(v[2]);
      double px = v[0] / l1, py = v[1] / l1;
      if (v[2] < 0.0) {
        double fx = (1.0 - fabs(py)) * sgn_nonneg(px);
        double fy = (1.0 - fabs(px)) * sgn_nonneg(py);
        px = fx; py = fy;
      }
      if (px > 1.0) px = 1.0;
      if (px < -1.0) px = -1.0;
      if (py > 1.0) py = 1.0;
      if (py < -1.0) py = -1.0;
      double qx = floor(px * 32767.0 + 0.5), qy = floor(py * 32767.0 + 0.5);
      double dx = qx / 32767.0, dy = qy / 32767.0;
      double vz = 1.0 - fabs(dx) - fabs(dy);
      double vx = dx, vy = dy;
      if (vz < 0.0) {
        vx = (1.0 - fabs(dy)) * sgn_nonneg(dx);
        vy = (1.0 - fabs(dx)) * sgn_nonneg(dy);
      }
      double n = sqrt(vx * vx + vy * vy + vz * vz);
      v[0] = vx / n; v[1] = vy / n; v[2] = vz / n;
      return;
    }
    case ORC_CODEC_YX4: {
      /* the paper's packing (Sec. 3.3): binary32 s_y and binary32 s_x + 4 sign(s_z)
         (sign(0) = +1); decoded with s_z = sign sqrt(1 - s_x^2 - s_y^2) */
      double y = (double)(float)v[1];
      double p = (double)(float)(v[0] + (v[2] >= 0.0 ? 4.0 : -4.0));
      double sg = p > 2.0 ? 1.0 : -1.0;
      double x = p - 4.0 * sg;
      double r = 1.0 - x * x - y * y;
      v[0] = x;
      v[1] = y;
      v[2] = sg * sqrt(r > 0.0 ? r : 0.0);
      return;
    }
    default:
      return;
  }
}

void orc_codec_roundtrip_many(double* v, long n, int codec) {
  for (long k = 0; k < n; ++k) orc_codec_roundtrip(v + 3 * k, codec);
}

static void normalize3(double v[3]) {
  double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  v[0] /= n; v[1] /= n; v[2] /= n;
}

/* ------------------------------------------------------------------------ */
/* Lattice helpers                                                           */
/* ------------------------------------------------------------------------ */
static long site_of(int L, int x, int y, int z) { return (long)x + (long)L * ((long)y + (long)L * z); }

static long neighbour(int L, long i, int axis, int dir) {
  int x = (int)(i % L), y = (int)((i / L) % L), z = (int)(i / ((long)L * L));
  int* c = axis == 0 ? &x : (axis == 1 ? &y : &z);
  *c = (*c + dir + L) % L;
  return site_of(L, x, y, z);
}

static int parity_of(int L, long i) {
  int x = (int)(i % L), y = (int)((i / L) % L), z = (int)(i / ((long)L * L));
  return (x + y + z) & 1;
}

/* Random initial state: cos(theta) = 2 u1 - 1, phi = 2 pi u2 (uniform on S^2) */
void orc_init_spins(double* s, int L, int W, uint64_t sys_base, uint64_t seed, int codec) {
  long N = (long)L * L * L;
  for (int w = 0; w < W; ++w) {
    for (long i = 0; i < N; ++i) {
      double u1, u2;
      pair_uniforms((uint32_t)i, sys_base + (uint64_t)w, 0u, ORC_TAG_INIT, seed, &u1, &u2);
      double z = 2.0 * u1 - 1.0;
      double rho = 2.0 * sqrt(u1 * (1.0 - u1));
      double phi = 2.0 * ORC_PI * u2;
      double* v = s + 3 * ((long)w * N + i);
      v[0] = rho * cos(phi);
      v[1] = rho * sin(phi);
      v[2] = z;
      orc_codec_roundtrip(v, codec);
    }
  }
}

/* Local molecular field of Eq. (2): h_i = sum_{j in nn(i)} J_ij s_j + H_i */
void orc_local_field(const double* s_sys, const double* J, const double* H, int L, long i,
                     double h[3]) {
  h[0] = h[1] = h[2] = 0.0;
  for (int a = 0; a < 3; ++a) {
    long ip = neighbour(L, i, a, +1);
    long im = neighbour(L, i, a, -1);
    double jp = J[3 * i + a];    /* bond (i, i + e_a) */
    double jm = J[3 * im + a];   /* bond (i - e_a, i) */
    for (int c = 0; c < 3; ++c) {
      h[c] += jp * s_sys[3 * ip + c];
      h[c] += jm * s_sys[3 * im + c];
    }
  }
  if (H) {
    for (int c = 0; c < 3; ++c) h[c] += H[3 * i + c];
  }
}

/* Over-relaxation, Eq. (3): reflect s at the local field, s' = 2 (s.h)/(h.h) h - s */
void orc_or_move(double s[3], const double h[3]) {
  double hh = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
  if (hh > 0.0) {
    double sh = s[0] * h[0] + s[1] * h[1] + s[2] * h[2];
    double f = 2.0 * sh / hh;
    for (int c = 0; c < 3; ++c) s[c] = f * h[c] - s[c];
  }
  normalize3(s);
}

/* Heat bath, Eq. (2): s' ~ exp(beta h.s) on the unit sphere.
   With a = beta |h| and t the angle to h, cos t has density a e^{a c} / (2 sinh a)
   on [-1, 1]; its inverse CDF gives d = 1 - cos t = -log(u + (1-u) e^{-2a}) / a,
   written as -log1p((1-u) expm1(-2a)) / a.  The azimuth is uniform. */
#define ORC_HB_A_MIN 1e-12
void orc_hb_move(double s[3], const double h[3], double beta, double u1, double u2) {
  double hn = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
  double a = beta * hn;
  double d;
  if (a > ORC_HB_A_MIN) {
    d = -log1p((1.0 - u1) * expm1(-2.0 * a)) / a;
  } else {
    d = 2.0 * (1.0 - u1);                     /* a -> 0: cos t uniform on [-1, 1] */
  }
  if (d < 0.0) d = 0.0;
  if (d > 2.0) d = 2.0;
  double ct = 1.0 - d;
  double st = sqrt(d * (2.0 - d));
  double phi = 2.0 * ORC_PI * u2;
  double cp = cos(phi), sp = sin(phi);
  double n[3];
  if (hn > 0.0) {
    n[0] = h[0] / hn; n[1] = h[1] / hn; n[2] = h[2] / hn;
  } else {
    n[0] = 0.0; n[1] = 0.0; n[2] = 1.0;
  }
  /* orthonormal frame (e1, e2, n): Duff et al., "Building an orthonormal
     basis, revisited", JCGT 6(1), 2017 */
  double sg = n[2] >= 0.0 ? 1.0 : -1.0;
  double A = -1.0 / (sg + n[2]);
  double B = n[0] * n[1] * A;
  double e1[3] = {1.0 + sg * n[0] * n[0] * A, sg * B, -sg * n[0]};
  double e2[3] = {B, sg + n[1] * n[1] * A, -n[1]};
  for (int c = 0; c < 3; ++c) s[c] = ct * n[c] + st * (cp * e1[c] + sp * e2[c]);
  normalize3(s);
}

void orc_hb_many(double* s, const double* h, const double* beta, const double* u1,
                 const double* u2, long n) {
  for (long k = 0; k < n; ++k) orc_hb_move(s + 3 * k, h + 3 * k, beta[k], u1[k], u2[k]);
}

/* One half-sweep: every site of the given parity, every system.  Sites of one
   parity have no bond between them, so their order does not matter. */
void orc_or_half(double* s, const double* J, const double* H, int L, int W, int parity,
                 int codec) {
  long N = (long)L * L * L;
#pragma omp parallel for schedule(static)
  for (int w = 0; w < W; ++w) {
    double* sw = s + 3 * (long)w * N;
    for (long i = 0; i < N; ++i) {
      if (parity_of(L, i) != parity) continue;
      double h[3];
      orc_local_field(sw, J, H, L, i, h);
      orc_or_move(sw + 3 * i, h);
      orc_codec_roundtrip(sw + 3 * i, codec);
    }
  }
}

void orc_hb_half(double* s, const double* J, const double* H, int L, int W, int parity,
                 const double* beta, uint64_t sys_base, uint64_t seed, uint32_t sweep,
                 int codec) {
  long N = (long)L * L * L;
#pragma omp parallel for schedule(static)
  for (int w = 0; w < W; ++w) {
    double* sw = s + 3 * (long)w * N;
    for (long i = 0; i < N; ++i) {
      if (parity_of(L, i) != parity) continue;
      double h[3], u1, u2;
      orc_local_field(sw, J, H, L, i, h);
      pair_uniforms((uint32_t)i, sys_base + (uint64_t)w, sweep, ORC_TAG_HB, seed, &u1, &u2);
      orc_hb_move(sw + 3 * i, h, beta[w], u1, u2);
      orc_codec_roundtrip(sw + 3 * i, codec);
    }
  }
}

/* Multi-hit tile schedule (Sec. 3.2, the double checkerboard; Table 1's
   "10 x (1 HB + 10 OR)").  The lattice is cut into cubic tiles of edge T
   (T even, L / T even), coloured by the parity of their tile coordinates, so
   that no two tiles of one colour share a bond.  For colour 0, then colour 1
   (the bits of `colors` select them), every tile of that colour is updated
   n_rounds times by n_or over-relaxation sweeps and then n_hb heat-bath
   sweeps of its own sites, while every spin outside it stays as it is; a
   tile sweep visits the tile's sites of parity 0, then those of parity 1.
   The k-th tile sweep of the call (k = 0 .. n_rounds (n_or + n_hb) - 1, in
   that order) draws its heat-bath numbers with sweep counter sweep0 + k.
   Tiles of one colour do not interact, so their order does not matter. */
void orc_multihit(double* s, const double* J, const double* H, int L, int W, int T, int colors,
                  int n_rounds, int n_or, int n_hb, const double* beta, uint64_t sys_base,
                  uint64_t seed, uint32_t sweep0, int codec) {
  const long N = (long)L * L * L;
  const int B = L / T, per_round = n_or + n_hb;
#pragma omp parallel for schedule(static)
  for (int w = 0; w < W; ++w) {
    double* sw = s + 3 * (long)w * N;
    for (int color = 0; color < 2; ++color) {
      if (!((colors >> color) & 1)) continue;
      for (int Z = 0; Z < B; ++Z)
        for (int Y = 0; Y < B; ++Y)
          for (int X = 0; X < B; ++X) {
            if (((X + Y + Z) & 1) != color) continue;
            for (int r = 0; r < n_rounds; ++r)
              for (int k = 0; k < per_round; ++k) {
                const int hb = k >= n_or;
                const uint32_t sweep = sweep0 + (uint32_t)(r * per_round + k);
                for (int parity = 0; parity < 2; ++parity)
                  for (int z = Z * T; z < Z * T + T; ++z)
                    for (int y = Y * T; y < Y * T + T; ++y)
                      for (int x = X * T; x < X * T + T; ++x) {
                        const long i = site_of(L, x, y, z);
                        if (parity_of(L, i) != parity) continue;
                        double h[3];
                        orc_local_field(sw, J, H, L, i, h);
                        if (hb) {
                          double u1, u2;
                          pair_uniforms((uint32_t)i, sys_base + (uint64_t)w, sweep, ORC_TAG_HB,
                                        seed, &u1, &u2);
                          orc_hb_move(sw + 3 * i, h, beta[w], u1, u2);
                        } else {
                          orc_or_move(sw + 3 * i, h);
                        }
                        orc_codec_roundtrip(sw + 3 * i, codec);
                      }
              }
          }
    }
  }
}

/* Eq. (1), each bond once: E = - sum_i sum_a J_i,a s_i.s_{i+e_a} - sum_i H_i.s_i */
void orc_energy(const double* s, const double* J, const double* H, int L, int W, double* E) {
  long N = (long)L * L * L;
#pragma omp parallel for schedule(static)
  for (int w = 0; w < W; ++w) {
    const double* sw = s + 3 * (long)w * N;
    double e = 0.0;
    for (long i = 0; i < N; ++i) {
      for (int a = 0; a < 3; ++a) {
        long j = neighbour(L, i, a, +1);
        double dot = sw[3 * i] * sw[3 * j] + sw[3 * i + 1] * sw[3 * j + 1] +
                     sw[3 * i + 2] * sw[3 * j + 2];
        e -= J[3 * i + a] * dot;
      }
      if (H) {
        e -= H[3 * i] * sw[3 * i] + H[3 * i + 1] * sw[3 * i + 1] + H[3 * i + 2] * sw[3 * i + 2];
      }
    }
    E[w] = e;
  }
}

/* Parallel tempering, Eq. (4): for each replica chain, pairs (k, k+1) from the
   lowest temperature up, accept with min[1, exp(dbeta dE)], dbeta = 1/T_{k+1} -
   1/T_k, dE = E_{k+1} - E_k; an accepted swap exchanges the temperatures of the
   two configurations (perm entries), so the walk carries a configuration upward. */
void orc_pt(const double* E, const double* temps, int32_t* perm, int R_O, int R_T,
            uint64_t chain_base, uint64_t seed, uint32_t pt_step, int32_t* accepted) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (int r = 0; r < R_O; ++r) {
    int32_t* pr = perm + (long)r * R_T;
    for (int k = 0; k + 1 < R_T; ++k) {
      int a = pr[k], b = pr[k + 1];
      double dbeta = 1.0 / temps[k + 1] - 1.0 / temps[k];
      double dE = E[(long)r * R_T + b] - E[(long)r * R_T + a];
      double x = dbeta * dE;
      uint32_t ctr[4] = {(uint32_t)k, (uint32_t)(chain_base + (uint64_t)r), pt_step, ORC_TAG_PT};
      uint32_t out[4];
      orc_philox4x32_10(ctr, key, out);
      double u = orc_uniform(out[0]);
      int acc = (x >= 0.0) || (u < exp(x));
      if (acc) {
        pr[k] = b;
        pr[k + 1] = a;
      }
      if (accepted) accepted[(long)r * (R_T - 1) + k] = acc;
    }
  }
}

/* Eq. (5) and its k-dependent form: q^{mu nu}(k) = (1/N) sum_i s_i^mu(1) s_i^nu(2) e^{i k.R_i}
   for the configurations of replicas 0 and 1 at each temperature slot t, with
   k = 0 (q) and k = (2 pi / L) e_a for a = x, y, z (qk[t][a][mu][nu][re, im]). */
void orc_measure(const double* s, int L, int R_T, const int32_t* perm, double* q,
                 double* qk) {
  long N = (long)L * L * L;
  /* temperature slots are independent: each keeps its own sums in site order */
#pragma omp parallel for schedule(static)
  for (int t = 0; t < R_T; ++t) {
    const double* sa = s + 3 * (long)perm[t] * N;
    const double* sb = s + 3 * ((long)R_T + perm[R_T + t]) * N;
    double acc[3][3] = {{0}};
    double acck[3][3][3][2] = {{{{0}}}};
    for (long i = 0; i < N; ++i) {
      int coord[3] = {(int)(i % L), (int)((i / L) % L), (int)(i / ((long)L * L))};
      /* e^{i k_a x_a} of this site for the three modes */
      double cs[3], sn[3];
      for (int a = 0; a < 3; ++a) {
        double arg = 2.0 * ORC_PI * (double)coord[a] / (double)L;
        cs[a] = cos(arg);
        sn[a] = sin(arg);
      }
      for (int mu = 0; mu < 3; ++mu) {
        for (int nu = 0; nu < 3; ++nu) {
          double p = sa[3 * i + mu] * sb[3 * i + nu];
          acc[mu][nu] += p;
          for (int a = 0; a < 3; ++a) {
            acck[a][mu][nu][0] += p * cs[a];
            acck[a][mu][nu][1] += p * sn[a];
          }
        }
      }
    }
    for (int mu = 0; mu < 3; ++mu)
      for (int nu = 0; nu < 3; ++nu) {
        q[(long)t * 9 + mu * 3 + nu] = acc[mu][nu] / (double)N;
        for (int a = 0; a < 3; ++a)
          for (int ri = 0; ri < 2; ++ri)
            qk[(((long)t * 3 + a) * 9 + mu * 3 + nu) * 2 + ri] = acck[a][mu][nu][ri] / (double)N;
      }
  }
}

/* Local chirality of one system: for each site i and lattice direction a,
   kappa = s_{i+a} . (s_i x s_{i-a}) with periodic neighbours (Sec. 2). */
void orc_chirality(const double* s, int L, double* kappa) {
  long N = (long)L * L * L;
  for (long i = 0; i < N; ++i) {
    int c[3] = {(int)(i % L), (int)((i / L) % L), (int)(i / ((long)L * L))};
    for (int a = 0; a < 3; ++a) {
      int cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
      cp[a] = (c[a] + 1) % L;
      cm[a] = (c[a] + L - 1) % L;
      long ip = cp[0] + (long)L * (cp[1] + (long)L * cp[2]);
      long im = cm[0] + (long)L * (cm[1] + (long)L * cm[2]);
      const double* u = s + 3 * ip;  /* s_{i+a} */
      const double* v = s + 3 * i;   /* s_i */
      const double* w = s + 3 * im;  /* s_{i-a} */
      double cross[3] = {v[1] * w[2] - v[2] * w[1], v[2] * w[0] - v[0] * w[2],
                         v[0] * w[1] - v[1] * w[0]};
      kappa[3 * i + a] = u[0] * cross[0] + u[1] * cross[1] + u[2] * cross[2];
    }
  }
}

/* Replica-pair spin and chiral overlaps at the modes k = 0, (2 pi/L) e_a, by
   direct summation in FP64 (the four-replica sums and the chiral overlap of
   Sec. 2). */
void orc_overlaps(const double* s, int L, int R_O, int R_T, const int32_t* perm, double* D,
                  double* C) {
  static const int PA[6] = {0, 0, 1, 0, 1, 2}, PB[6] = {1, 2, 2, 3, 3, 3};
  long N = (long)L * L * L;
  int r = R_O < 4 ? R_O : 4;
  int n_pairs = r * (r - 1) / 2;
  double* ka = (double*)malloc(sizeof(double) * 3 * N);
  double* kb = (double*)malloc(sizeof(double) * 3 * N);
  for (int t = 0; t < R_T; ++t) {
    for (int k = 0; k < n_pairs; ++k) {
      const double* sa = s + 3 * ((long)PA[k] * R_T + perm[PA[k] * R_T + t]) * N;
      const double* sb = s + 3 * ((long)PB[k] * R_T + perm[PB[k] * R_T + t]) * N;
      orc_chirality(sa, L, ka);
      orc_chirality(sb, L, kb);
      double accD[4][2] = {{0}}, accC[3][4][2] = {{{0}}};
      for (long i = 0; i < N; ++i) {
        int c[3] = {(int)(i % L), (int)((i / L) % L), (int)(i / ((long)L * L))};
        double ph[4][2] = {{1.0, 0.0}};
        for (int a = 0; a < 3; ++a) {
          double arg = 2.0 * ORC_PI * (double)c[a] / (double)L;
          ph[a + 1][0] = cos(arg);
          ph[a + 1][1] = sin(arg);
        }
        double d = sa[3 * i] * sb[3 * i] + sa[3 * i + 1] * sb[3 * i + 1] + sa[3 * i + 2] * sb[3 * i + 2];
        for (int m = 0; m < 4; ++m) {
          accD[m][0] += d * ph[m][0];
          accD[m][1] += d * ph[m][1];
          for (int a = 0; a < 3; ++a) {
            double pk = ka[3 * i + a] * kb[3 * i + a];
            accC[a][m][0] += pk * ph[m][0];
            accC[a][m][1] += pk * ph[m][1];
          }
        }
      }
      for (int m = 0; m < 4; ++m)
        for (int ri = 0; ri < 2; ++ri) {
          if (D) D[(((long)t * n_pairs + k) * 4 + m) * 2 + ri] = accD[m][ri] / (double)N;
          if (C)
            for (int a = 0; a < 3; ++a)
              C[((((long)t * n_pairs + k) * 3 + a) * 4 + m) * 2 + ri] = accC[a][m][ri] / (double)N;
        }
    }
  }
  free(ka);
  free(kb);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the later parallel loops (timing only: every loop is over
   independent systems or sites, so the results do not depend on it). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
