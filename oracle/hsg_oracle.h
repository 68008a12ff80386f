/*
 * FP64 CPU oracle for the Heisenberg spin-glass Monte Carlo method of
 * Yavors'kii & Weigel, "Optimized GPU simulation of continuous-spin glass
 * models" (arXiv:1204.6192).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header,
 * table or constant with the CUDA library; both sides implement the Philox
 * generator from its published definition (Salmon et al., SC'11).
 *
 * Conventions (identical meaning on both sides, written out independently):
 *   lattice     L^3 periodic, L even, site i = x + L*(y + L*z),
 *               parity p(i) = (x + y + z) mod 2
 *   spins       s[w][i][c], W systems, c = 0,1,2 (x, y, z components)
 *   couplings   J[i][a]: bond between i and i + e_a, a = 0,1,2
 *   field       H[i][c]
 *   system      w = r * n_temps + j  (replica r, memory slot j)
 *   perm        perm[r][t] = memory slot j that holds temperature t
 *   Philox key  (seed & 0xffffffff, seed >> 32)
 *   Philox ctr  init : (i, gsys >> 1, 0, 0)      words 2*(gsys&1), +1
 *               heat : (i, gsys >> 1, sweep, 1)  words 2*(gsys&1), +1
 *               PT   : (k, gchain, pt_step, 2)   word 0
 *   uniform     u(x) = (2*(x >> 9) + 1) * 2^-24, in (0, 1), exact in FP32/FP64
 *
 * Parity pins: every function is checked by tests/test_oracle_*.py against
 * invariants, closed forms, brute force or an independent library routine.
 */
#ifndef HSG_ORACLE_H
#define HSG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_TAG_INIT = 0, ORC_TAG_HB = 1, ORC_TAG_PT = 2 };
enum { ORC_CODEC_NONE = 0, ORC_CODEC_FP16 = 1, ORC_CODEC_BF16 = 2,
       ORC_CODEC_ANGLE16 = 3, ORC_CODEC_OCT16 = 4,
       ORC_CODEC_FP32 = 5, ORC_CODEC_YX4 = 6 };

void   orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void   orc_philox_many(const uint32_t* ctr, long n, uint64_t seed, uint32_t* out);
double orc_uniform(uint32_t x);

/* storage rounding of one spin vector, in place (the codec's encode + decode) */
void   orc_codec_roundtrip(double v[3], int codec);
double orc_round_fp16(double x);
double orc_round_bf16(double x);
void   orc_codec_roundtrip_many(double* v, long n, int codec);

void   orc_init_spins(double* s, int L, int W, uint64_t sys_base, uint64_t seed, int codec);
void   orc_local_field(const double* s_sys, const double* J, const double* H, int L, long i,
                       double h[3]);
void   orc_or_move(double s[3], const double h[3]);
void   orc_hb_move(double s[3], const double h[3], double beta, double u1, double u2);
void   orc_hb_many(double* s, const double* h, const double* beta, const double* u1,
                   const double* u2, long n);

void   orc_or_half(double* s, const double* J, const double* H, int L, int W, int parity,
                   int codec);
void   orc_hb_half(double* s, const double* J, const double* H, int L, int W, int parity,
                   const double* beta, uint64_t sys_base, uint64_t seed, uint32_t sweep,
                   int codec);
/* Multi-hit tile schedule (Sec. 3.2, Table 1): tiles of edge T coloured by the
   parity of their tile coordinates; per colour, every tile gets n_rounds x
   (n_or OR + n_hb HB) tile sweeps with the rest of the lattice fixed; the
   k-th tile sweep keys its heat-bath numbers with sweep0 + k.  colors: bit 0
   colour 0, bit 1 colour 1.  T even, L / T even. */
void   orc_multihit(double* s, const double* J, const double* H, int L, int W, int T, int colors,
                    int n_rounds, int n_or, int n_hb, const double* beta, uint64_t sys_base,
                    uint64_t seed, uint32_t sweep0, int codec);
void   orc_energy(const double* s, const double* J, const double* H, int L, int W, double* E);
void   orc_pt(const double* E, const double* temps, int32_t* perm, int R_O, int R_T,
              uint64_t chain_base, uint64_t seed, uint32_t pt_step, int32_t* accepted);
void   orc_measure(const double* s, int L, int R_T, const int32_t* perm, double* q,
                   double* qk);
/* Local chirality (Sec. 2, three spins on a line): kappa[i][a] =
   s_{i+a} . (s_i x s_{i-a}) for a = x, y, z, one system s[N][3]. */
void   orc_chirality(const double* s, int L, double* kappa);
/* Replica-pair overlaps at slot t for pairs (a, b) of the first min(R_O, 4)
   replicas, in the order (0,1) (0,2) (1,2) (0,3) (1,3) (2,3) (the pairs of
   the first r replicas come first):
   D[t][pair][m][re,im] = (1/N) sum_i (s_i^A . s_i^B) e^{i k_m.R_i} and
   C[t][pair][alpha][m][re,im] = (1/N) sum_i kappa_i^{alpha,A} kappa_i^{alpha,B} e^{i k_m.R_i},
   k_0 = 0, k_{1,2,3} = (2 pi / L) e_{x,y,z}.  Either output may be NULL. */
void   orc_overlaps(const double* s, int L, int R_O, int R_T, const int32_t* perm, double* D,
                    double* C);
int    orc_num_threads(void);
void   orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
