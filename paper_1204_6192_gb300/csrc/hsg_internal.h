// Internal layout and kernel-launch interface of libhsg (not part of the C ABI).
//
// Device data layout (all samples of a context in one allocation each):
//   spins   per sample, sites in parity-split order: storage site
//           ss(i) = p(i) * N/2 + (i >> 1), so each half-sweep touches one
//           contiguous half of the array.  Systems come in chunks of 4: chunk g
//           holds systems 4g .. 4g+3 of one site (16 bytes for FP32 and the
//           packed 32-bit formats, 8 bytes for FP16/BF16).  Layout
//           [plane c][chunk g][ss][4 systems]: component formats have three
//           planes (x, y, z), packed formats one.  Consecutive sites of one
//           chunk are contiguous, so a warp of consecutive sites reads 256-512
//           contiguous bytes, and one thread can walk the chunks of its site.
//   records per storage site 12 scalars (FP32 or FP16):
//           [J+x, J-x, J+y, J-y], [J+z, J-z, Hx, Hy], [Hz, 0, 0, 0]
//           i.e. the six bonds of the site and its field, shared by all Wp
//           systems of the sample (the paper's reuse of J and H across
//           temperatures and replicas, Sec. 3.3).
//   beta    float [n_samples][Wp]: inverse temperature of each system.
//   perm    int32 [n_samples][R_O][R_T]; temps/inv_temps double [n_samples][R_T].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hsg {

// spin storage formats (values of hsg_precision)
enum Fmt { FMT_F32 = 0, FMT_F16 = 1, FMT_BF16 = 2, FMT_ANG16 = 3, FMT_OCT16 = 4, FMT_YX4 = 5 };

constexpr int SWEEP_BS = 256;
constexpr int MAX_E_SPLITS = 256;   // first-level units per sample of the energy sums     // threads per block, streaming sweep kernels
constexpr int RED_BS = SWEEP_BS;  // energy kernel: same blocks as the sweep

struct FastDivH {
  uint32_t d, m, s;
};

struct SampleDev {
  int L, N, Lh;
  uint32_t fdLh_m, fdLh_s, fdL_m, fdL_s;
  long long spin_off;       // byte offset of the sample's spin block
  long long plane_stride;   // bytes between component planes (N * Wp * ELEM)
  long long rec_off;        // record index of storage site 0
  int sys_base;             // global id of system 0 = sample * Wp
  int blk0, blk1;           // the sample's blocks in the sweep block table
  // packed formats: the opposite parity decoded to binary32 before each
  // half-sweep, chunk layout [c][g][N/2][4] (byte offset and plane stride)
  long long dec_off, dec_plane_stride;
};

struct SweepParams {
  unsigned char* spins;
  const void* rec;
  const SampleDev* samples;
  const int4* blocks;       // (sample, chunk group, first half-site) per block
  const float* beta;        // [n_samples][Wp]
  const unsigned long long* counters;   // [n_samples][2]: sweeps done, PT passes done
  const unsigned char* active;          // [n_samples]: 0 = the sample is frozen
  int G, Wp, GPT;            // chunks per site, padded systems, chunks per thread
  uint32_t seed_lo, seed_hi;
  int parity;
  int sweep_offset;
  double* epart;            // energy partials [2][n_blocks][Wp] (energy variant only)
  int n_blocks;
  int blk_base;             // block table entry of launch block 0 (a pass's first block)
  int n_launch;             // blocks of this launch
  int reverse;              // nonzero: launch block k runs table entry blk_base + n_launch - 1 - k
                            // (so a launch starts on the planes the previous one ended with)
  uint32_t rk[20];          // Philox round keys of the seed
  const unsigned char* dec; // packed formats: the opposite parity as binary32 (see SampleDev)
  // staged sweeps (hsg_wave.cu): bytes of one stage of neighbour rows, offset of
  // stage 0 in dynamic shared memory, the error word of their bounded waits
  int stage_bytes, stage_off;
  unsigned int* err;
  unsigned long long timeout_ns;
  unsigned int* bounds_err;  // HSG_CHECK builds: set when a device bounds check fails
};

// Device bounds checks of the sweep kernels, compiled in with -DHSG_CHECK: a
// check that fails records it in an error word (the host reports HSG_ESTATE)
// and the caller skips the access; nothing traps.  Without HSG_CHECK the
// condition is not evaluated and the access goes ahead.
#ifdef HSG_CHECK
#define HSG_OUT_OF_BOUNDS(cond, errword) (!(cond) ? (atomicExch((errword), 1u), true) : false)
#else
#define HSG_OUT_OF_BOUNDS(cond, errword) false
#endif

struct EnergyParams {
  const unsigned char* spins;
  const void* rec;
  const SampleDev* samples;
  const int4* blocks;       // the sweep block table
  double* partials;         // [2][n_blocks][Wp]: even-site and odd-site terms per block
  double* partials2;        // [n_samples][splits][Wp]: second reduction level
  double* E;                // [n_samples][Wp]
  const unsigned char* active;   // [n_samples]: frozen samples keep their energies
  int G, Wp, GPT, n_samples, n_blocks, splits;
};

struct PTParams {
  const double* E;          // [n_samples][Wp]
  const double* inv_temps;  // [n_samples][R_T]
  int* perm;                // [n_samples][R_O][R_T]
  float* beta;              // [n_samples][Wp]
  unsigned long long* accepted;   // [n_samples][R_O][R_T-1]
  unsigned long long* moved;      // [n_samples][R_O][R_T]: passes after which the slot's configuration moved
  unsigned char* tstate;          // [n_samples][R_O][R_T] by memory slot: 0 none, 1 last end T_1, 2 then T_R
  unsigned int* tunnel;           // [n_samples][R_O][R_T] by memory slot: closed loops T_1 -> T_R -> T_1
  unsigned long long* counters;   // [n_samples][2]: sweeps done, PT passes done
  const unsigned char* active;    // [n_samples]: frozen samples are skipped
  int n_samples, R_O, R_T, Wp;
  uint32_t seed_lo, seed_hi;
  int sweeps_per_call;      // added to each active sample's sweep counter after the pass
  int bump_pt;              // 1: this is a PT pass (each active sample's PT counter += 1)
};


// Replica-pair measurements (hsg_overlap.cu): the overlap tensor of replicas
// 0 and 1 (one unit) or the scalar / chiral overlaps of n_pairs replica pairs.
struct OverlapParams {
  const unsigned char* spins;
  const SampleDev* samples;
  const int* perm;
  double* partials;         // [n_samples][n_pairs][n_tiles][R_T][values]
  double* D;                // q [ns][R_T][3][3], or D [ns][R_T][n_pairs][4][2]; may be null
  double* C;                // qk [ns][R_T][3][3][3][2], or C [ns][R_T][n_pairs][3][4][2]; may be null
  int n_samples, R_O, R_T, Wp, n_pairs, n_tiles;
  // staged kernels only (sub > 0): storage sites per stage and per block, chunk
  // groups staged, padded bytes per staged (plane, group) row; bounded waits
  int sub, tile_ss, Gu, grow;
  unsigned int* err;        // set when a wait for a staged copy ran out
  unsigned long long timeout_ns;
};
constexpr int MEAS_BS = 256;       // threads per block of the measurement kernels
constexpr int MEAS_TILE = 1024;    // sites per block of the direct (unstaged) kernels
// FP64 partial values per (unit, tile, slot) of the direct kernels: 21 per
// tensor row, 28 (7 without chirality) per pair
int meas_partial_values(bool qtensor, bool chiral);

// Geometry of the staged kernels (tensor q(k) and scalar pair overlaps): the
// spins of a block's run of storage sites reach shared memory by bulk copies
// in stages of `sub` sites.  ok = 0 when even 8 sites of the staged systems do
// not fit; the direct kernels serve that case.
struct StagedGeom {
  int ok, sub, tile_ss, Gu, grow, n_tiles, rounds, smem, values;
};
StagedGeom staged_geometry(int fmt, bool qtensor, int R_O, int R_T, long long n_max,
                           long long n_total);

// Chiral overlaps in two stages: the chirality of every site into a binary32
// buffer in the chunk layout ([a][g][ss][4], g < Gu), then the staged kernel
// over that buffer.
struct ChiralityParams {
  const unsigned char* spins;
  unsigned char* kappa;
  const SampleDev* samples;     // the spins' sample table
  const SampleDev* ksamples;    // the same samples with the buffer's offsets and plane strides
  const int4* blocks;           // the sweep block table
  int G, GPT, Gu, parity;
};
cudaError_t launch_chirality(int fmt, const ChiralityParams& p, int n_blocks, cudaStream_t st);
cudaError_t launch_chiral_staged(const OverlapParams& p, cudaStream_t st);

struct ConvParams {
  unsigned char* spins;
  const SampleDev* samples;
  const int4* blocks;       // (sample, chunk g, first site) per block, all sites
  float* xyz;               // [sum_s W * N_s * 3]
  const long long* xyz_off; // per sample, float offset of its block
  int G, Wp, W;
  uint32_t fdG_m, fdG_s;
  uint32_t seed_lo, seed_hi;
};

struct PersistParams {
  SweepParams sw;           // parity and sweep offset set per phase inside the kernel
  EnergyParams en;
  PTParams pt;
  unsigned int* bar;        // [0] arrivals, [1] generation, [2] error word
  unsigned long long timeout_ns;
  int n_steps, nhb, nor;
  int drop_first;           // fault injection: block 0 skips the first barrier
  const int* pass_bound;    // [n_passes + 1]: block table range of each pass
  int n_passes;
};

// Multi-hit tile updates (hsg_multihit.cu): one launch per tile colour.
struct MultihitParams {
  unsigned char* spins;
  const void* rec;
  const SampleDev* samples;
  const int4* blocks;       // (sample, tile, chunk group, 0); colour 0 tiles first
  const float* beta;        // [n_samples][Wp]
  const unsigned long long* counters;   // [n_samples][2]: sweeps done, PT passes done
  const unsigned char* active;          // [n_samples]
  int Wp;
  int n_rounds, n_or, n_hb;             // per tile: n_rounds x (n_or OR + n_hb HB) tile sweeps
  int blk_base;             // block table entry of launch block 0
  uint32_t rk[20];          // Philox round keys of the seed
};
cudaError_t launch_multihit(int fmt, bool j16, bool fast, int tile, const MultihitParams& p,
                            int n_blocks, cudaStream_t st);

// Fused over-relaxation sweep (hsg_fused.cu): one launch per sweep, reading
// `src` and writing `dst` (two spin buffers of the same layout).  A work item
// is one column: (sample, chunk group, y0 | ny << 16, za | zb << 16) -- the band
// of rows [y0, y0 + ny) (ny = L: the whole plane) over the planes [za, zb).
constexpr int FUSED_CONSUMER_WARPS = 32;
constexpr int FUSED_THREADS = FUSED_CONSUMER_WARPS * 32;
constexpr int FUSED_SMEM_HEAD = 384;     // mbarriers, the abort flag and the two copy cursors
constexpr int FUSED_ODD_SLOTS = 6, FUSED_EVEN_SLOTS = 5;
constexpr int FUSED_SITES_PER_THREAD = 1;                        // per step (even + odd sites)
constexpr int FUSED_MAX_SITES = FUSED_SITES_PER_THREAD * FUSED_THREADS;
struct FusedParams {
  const unsigned char* src;
  unsigned char* dst;
  const void* rec;
  const SampleDev* samples;
  const int4* items;
  const unsigned char* active;          // [n_samples]: frozen samples are skipped
  int n_items;
  uint32_t slot1, slot0;                // bytes of one odd / even plane slot
  unsigned int* err;                    // set when a bounded wait ran out
  unsigned long long timeout_ns;
};
cudaError_t prepare_fused(int fmt, bool j16, size_t smem, int* blocks_per_sm);
cudaError_t launch_fused(int fmt, bool j16, const FusedParams& p, int grid, size_t smem,
                         cudaStream_t st);

// Wavefront over-relaxation sweep (hsg_wave.cu): both half-sweeps of one pass
// in one launch of 2 (b1 - b0) blocks, odd blocks trailing the even blocks of
// their planes (see the file).
struct WaveParams {
  SweepParams sw;           // parity set per block
  const int* order;         // [2 n_blocks]: per ticket, (block << 1) | parity; a pass's tickets at 2 b0
  const int4* deps;         // [n_blocks]: for an odd block, even blocks [x, y) and [z, w) it waits for
  unsigned int* flags;      // [n_blocks]: completion flag of each even block (epoch + 1)
  unsigned int* state;      // [0] tickets taken, [1] blocks finished, [2] epoch
  unsigned int* err;        // set when a wait ran out
  unsigned long long timeout_ns;
  int t0, n_tickets;        // this launch's tickets: order[t0 .. t0 + n_tickets)
  // fault injection (tests only): odd block `inject_block` (-1: none) also waits
  // for flags[never], which no block sets
  int inject_block, never;
};
bool fmt_has_wave(int fmt);
// Staged sweeps: every block copies the opposite-parity rows its sites read
// (plane z: rows y0-1 .. y0+R, planes z-1 and z+1: rows y0 .. y0+R-1; R = 256 /
// (L/2)) into a two-stage shared-memory ring with cp.async.bulk, one chunk group
// per stage.  Possible for every sample with L a power of 2, L >= 32.
constexpr int STAGED_STAGES = 2;
constexpr int STAGED_HEAD = 256;          // mbarriers and stage counters
bool lattice_has_staged(int L);
int staged_stage_bytes(int fmt, int Lh_max);
size_t staged_smem(int fmt, int gpt, bool energy, int Lh_max, int* stage_off);
// blocks per SM of the wave kernel (staged: with that dynamic shared memory)
cudaError_t wave_occupancy(int fmt, bool j16, bool staged, size_t smem, int* blocks_per_sm);
cudaError_t launch_wave(int fmt, bool j16, bool energy, bool staged, const WaveParams& p, size_t smem,
                        cudaStream_t st);
// one half-sweep (p.parity) of over-relaxation with the staged block body
cudaError_t launch_staged_half(int fmt, bool j16, bool energy, const SweepParams& p, int n_blocks,
                               size_t smem, cudaStream_t st);

// The packed spin formats (one or two 32-bit words per system) decode each
// neighbour spin once into a binary32 buffer before a half-sweep instead of
// at every one of its six uses.
inline bool fmt_decodes_once(int fmt) { return fmt == FMT_ANG16 || fmt == FMT_OCT16 || fmt == FMT_YX4; }

// launchers (hsg_kernels*.cu).  dec: the half-sweep reads its neighbours from
// p.dec, which launch_decode_parity filled with parity 1 - p.parity.
cudaError_t launch_half_sweep(int fmt, bool hb, bool j16, bool fast, bool energy, bool dec,
                              const SweepParams& p, int n_blocks, cudaStream_t st);
cudaError_t launch_decode_parity(int fmt, const SweepParams& p, int parity, int n_blocks,
                                 cudaStream_t st);
cudaError_t launch_energy(int fmt, bool j16, const EnergyParams& p, cudaStream_t st);
cudaError_t launch_energy_final(const EnergyParams& p, cudaStream_t st);
cudaError_t launch_pt(const PTParams& p, cudaStream_t st);
// The energy sums' last level and the PT pass of a step: one launch after the
// level-1 sums when samples x systems <= ENERGY_PT_FOLD_SYSTEMS, else two.
constexpr long long ENERGY_PT_FOLD_SYSTEMS = 4096;
bool energy_pt_folded(int n_samples, int Wp);
cudaError_t launch_energy_final_pt(const EnergyParams& e, const PTParams& p, cudaStream_t st);
// counters of the active samples += (sweeps, pts)
cudaError_t launch_bump(unsigned long long* counters, const unsigned char* active, int n_samples,
                        int sweeps, int pts, cudaStream_t st);
cudaError_t launch_overlaps(int fmt, const OverlapParams& p, bool chiral, cudaStream_t st);
// q^{mu nu}(k) of replicas 0 and 1: p.D = q, p.C = qk, partials [ns][R_T][3][n_blocks][21]
cudaError_t launch_qtensor(int fmt, const OverlapParams& p, cudaStream_t st);
cudaError_t launch_init(int fmt, const ConvParams& p, int n_blocks, cudaStream_t st);
cudaError_t launch_philox(const uint4* ctr, long long n, const SweepParams& p, uint4* out,
                          cudaStream_t st);
cudaError_t max_persistent_grid(int fmt, bool j16, bool fast, size_t smem, int* grid);
cudaError_t launch_persistent(int fmt, bool j16, bool fast, const PersistParams& P, int grid,
                              size_t smem, cudaStream_t st);
cudaError_t launch_get(int fmt, const ConvParams& p, int n_blocks, cudaStream_t st);
cudaError_t launch_set(int fmt, const ConvParams& p, int n_blocks, cudaStream_t st);

}  // namespace hsg
