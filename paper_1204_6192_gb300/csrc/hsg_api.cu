// Host runtime of libhsg: argument checking, device layout and allocation,
// kernel schedules for sweeps, steps (captured into a CUDA graph), parallel
// tempering and measurements, and the C ABI declared in include/hsg.h.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hsg.h"
#include "hsg_internal.h"

using namespace hsg;

namespace {

thread_local std::string g_create_error;

}  // namespace

struct hsg_ctx {
  hsg_options opt{};
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int fmt = 0, VEC = 4, PL = 3, ELEM = 4;
  bool j16 = false;
  int ns = 0, R_T = 0, R_O = 0, W = 0, Wp = 0, G = 0;
  int Lmax = 0;
  long long total_sites = 0;
  std::vector<int> L;
  std::vector<SampleDev> sd;
  uint32_t seed_lo = 0, seed_hi = 0;
  uint32_t fdG_m = 0, fdG_s = 0;

  // device state
  unsigned char* spins = nullptr;
  size_t spin_bytes = 0;
  // packed formats: the opposite parity decoded to binary32 before each half-sweep
  bool dec_once = false;
  unsigned char* dec = nullptr;
  size_t dec_bytes = 0;
  void* rec = nullptr;
  size_t rec_bytes = 0;
  SampleDev* d_sd = nullptr;
  int4* d_sweep_blocks = nullptr;     // (sample, chunk group, first half-site)
  int n_sweep_blocks = 0;
  int GPT = 1;                        // chunks per thread in the sweep kernels
  int4* d_conv_blocks = nullptr;      // (sample, chunk, first site)
  int n_conv_blocks = 0;
  double* d_epart = nullptr;        // energy partials [2][n_sweep_blocks][Wp]
  double* d_epart2 = nullptr;       // second level [n_samples][e_splits][Wp]
  int e_splits = 1;
  float* d_beta = nullptr;
  double* d_temps = nullptr;
  double* d_inv_temps = nullptr;
  int* d_perm = nullptr;
  double* d_E = nullptr;
  unsigned long long* d_acc = nullptr;
  unsigned long long* d_moved = nullptr;   // PT diagnostics [ns][R_O][R_T]
  unsigned char* d_tstate = nullptr;
  unsigned int* d_tunnel = nullptr;
  uint64_t seed = 0;
  uint64_t shape_hash = 0;            // lattice sizes, temperatures and records (checkpoints)
  unsigned long long* d_counters = nullptr;   // [ns][2]: sweeps done, PT passes done
  unsigned char* d_active = nullptr;          // [ns]: 0 = sample frozen
  double* d_mpart = nullptr;
  double* d_opart = nullptr;          // overlap partials (allocated at first use)
  bool e_valid = false;               // d_E holds the energies of the current state
  double* d_D = nullptr;
  double* d_C = nullptr;
  unsigned char* d_kappa = nullptr;   // chiralities, binary32 chunk layout (at first use)
  SampleDev* d_sd_k = nullptr;        // the sample table with the chirality buffer's offsets
  double* d_q = nullptr;
  double* d_qk = nullptr;
  float* d_xyz = nullptr;
  long long* d_xyz_off = nullptr;
  long long xyz_floats = 0;
  std::vector<long long> xyz_off;

  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;

  // persistent schedule
  int variant = HSG_VARIANT_TWO_PASS;   // resolved step schedule
  bool tune_pending = false;            // automatic schedule not yet tuned
  long long max_sweep_blocks = 0;       // sweep table capacity (one chunk per thread)
  unsigned int* d_bar = nullptr;        // grid barrier: arrivals, generation, error word; [3] measurement error word; [4] fused sweep error word; [5] wave and staged sweep error word; [6] device bounds checks (HSG_CHECK builds)
  int persist_grid = 0;
  size_t persist_smem = 0;
  bool inject_fault = false;

  // system-blocked passes: a step sweeps one range of the block table (a group
  // of systems) through all its sweeps before the next range
  // multi-hit tile schedule: block tables (sample, tile, chunk group), colour 0
  // first, built at first use for tile edges 4 and 8
  int4* d_mh_blocks[2] = {nullptr, nullptr};
  int mh_count[2][2] = {{0, 0}, {0, 0}};

  // fused over-relaxation sweep: a second spin buffer (each fused sweep reads
  // one buffer and writes the other; sweeps run in pairs, so the state is back
  // in `spins` after every call), the work items and the launch shape
  bool fused_possible = false;          // format and lattice sizes allow it
  bool use_fused = false;               // resolved choice of the schedule
  unsigned char* spins2 = nullptr;
  int4* d_fused_items = nullptr;
  int n_fused_items = 0, fused_grid = 0;
  size_t fused_smem = 0;
  uint32_t fused_slot1 = 0, fused_slot0 = 0;
  std::vector<int> fused_ny;            // band rows per sample

  // wave over-relaxation sweep: both half-sweeps in one launch of the sweep
  // block table's blocks, odd blocks trailing the even blocks of their planes
  bool wave_possible = false;           // the storage format allows it
  bool use_wave = false;                // resolved choice of the schedule
  // staged sweeps: neighbour rows through a shared-memory ring (the block body
  // of the wave sweep where possible, or of two half-sweep launches)
  bool staged_possible = false;         // format and every L allow it
  bool use_staged = false;              // HSG_SWEEP_STAGED in use
  int Lh_max = 0;
  int wave_lag = 0;                     // lag in use (even blocks)
  int* d_wave_order = nullptr;          // [2 max_sweep_blocks] ticket order of every pass
  int4* d_wave_deps = nullptr;          // [max_sweep_blocks] even-block ranges of each odd block
  unsigned int* d_wave_flags = nullptr; // [max_sweep_blocks] completion flags of the even blocks
  unsigned int* d_wave_state = nullptr; // tickets taken, blocks finished, epoch

  std::vector<int> pass_bound{0, 0};    // [n_passes + 1] block table bounds
  int* d_pass_bound = nullptr;
  long long pass_bytes = 0;             // resolved footprint bound (0: one pass)
  int max_passes = 1;

  hsg_status err = HSG_OK;
  std::string msg;
  std::vector<void*> allocations;
  int alloc_count = 0;                  // device allocations made
  int alloc_fail_at = 0;                // fault injection: fail this allocation (1-based; 0: off)
};

namespace {

hsg_status fail(hsg_ctx* c, hsg_status st, const std::string& m) {
  if (c) {
    if (c->err == HSG_OK) {
      c->err = st;
      c->msg = m;
    }
  } else {
    g_create_error = m;
  }
  return st;
}

// argument errors are not sticky
hsg_status bad_arg(hsg_ctx* c, const std::string& m) {
  if (c) c->msg = m;
  else g_create_error = m;
  return HSG_EINVAL;
}

#define HSG_CUDA(ctx, call)                                                             \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? HSG_ENOMEM : HSG_ECUDA,      \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

#define HSG_CHECK_CTX(ctx)                      \
  do {                                          \
    if (!(ctx)) return HSG_EINVAL;              \
    if ((ctx)->err != HSG_OK) return (ctx)->err; \
  } while (0)

// An NVTX range named after the API call for the duration of the host call
// (the GPU work it enqueues shows under it in a profiler's timeline; without
// a profiler attached a push and pop are a few instructions).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

void fastdiv(uint32_t d, uint32_t* m, uint32_t* s) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  *m = (uint32_t)((((1ull << l) - d) << 32) / d + 1ull);
  *s = l;
}

template <typename T>
hsg_status dev_alloc(hsg_ctx* c, T** p, size_t bytes) {
  if (c->alloc_fail_at > 0 && ++c->alloc_count == c->alloc_fail_at)
    return fail(c, HSG_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + "): injected allocation failure");
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) {
    return fail(c, HSG_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " +
                                   cudaGetErrorString(e));
  }
  c->allocations.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return HSG_OK;
}

#define HSG_TRY(expr)                  \
  do {                                 \
    hsg_status s_ = (expr);            \
    if (s_ != HSG_OK) return s_;       \
  } while (0)

int fmt_vec(int) { return 4; }
int fmt_planes(int f) { return (f == FMT_ANG16 || f == FMT_OCT16) ? 1 : (f == FMT_YX4 ? 2 : 3); }
int fmt_elem(int f) { return (f == FMT_F16 || f == FMT_BF16) ? 2 : 4; }

SweepParams sweep_params(hsg_ctx* c, int parity, int sweep_offset) {
  SweepParams p;
  p.spins = c->spins;
  p.rec = c->rec;
  p.samples = c->d_sd;
  p.blocks = c->d_sweep_blocks;
  p.beta = c->d_beta;
  p.counters = c->d_counters;
  p.active = c->d_active;
  p.G = c->G;
  p.Wp = c->Wp;
  p.GPT = c->GPT;
  p.seed_lo = c->seed_lo;
  p.seed_hi = c->seed_hi;
  p.parity = parity;
  p.sweep_offset = sweep_offset;
  p.epart = c->d_epart;
  p.n_blocks = c->n_sweep_blocks;
  p.blk_base = 0;
  p.n_launch = c->n_sweep_blocks;
  p.reverse = 0;
  p.dec = c->dec;
  p.stage_bytes = c->staged_possible ? staged_stage_bytes(c->fmt, c->Lh_max) : 0;
  p.stage_off = 0;
  p.err = c->d_bar + 5;
  p.bounds_err = c->d_bar + 6;
  p.timeout_ns = (unsigned long long)std::max(1, c->opt.barrier_timeout_ms) * 1000000ull;
  uint32_t k0 = c->seed_lo, k1 = c->seed_hi;
  for (int r = 0; r < 10; ++r) {
    p.rk[2 * r] = k0;
    p.rk[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return p;
}

EnergyParams energy_params(hsg_ctx* c) {
  EnergyParams p;
  p.spins = c->spins;
  p.rec = c->rec;
  p.samples = c->d_sd;
  p.blocks = c->d_sweep_blocks;
  p.partials = c->d_epart;
  p.partials2 = c->d_epart2;
  p.active = c->d_active;
  p.splits = c->e_splits;
  p.E = c->d_E;
  p.G = c->G;
  p.Wp = c->Wp;
  p.n_samples = c->ns;
  p.n_blocks = c->n_sweep_blocks;
  p.GPT = c->GPT;
  return p;
}

PTParams pt_params(hsg_ctx* c, int sweeps_per_call, int bump_pt) {
  PTParams p;
  p.E = c->d_E;
  p.inv_temps = c->d_inv_temps;
  p.perm = c->d_perm;
  p.beta = c->d_beta;
  p.accepted = c->d_acc;
  p.moved = c->d_moved;
  p.tstate = c->d_tstate;
  p.tunnel = c->d_tunnel;
  p.counters = c->d_counters;
  p.active = c->d_active;
  p.n_samples = c->ns;
  p.R_O = c->R_O;
  p.R_T = c->R_T;
  p.Wp = c->Wp;
  p.seed_lo = c->seed_lo;
  p.seed_hi = c->seed_hi;
  p.sweeps_per_call = sweeps_per_call;
  p.bump_pt = bump_pt;
  return p;
}

ConvParams conv_params(hsg_ctx* c, float* xyz, const long long* xyz_off) {
  ConvParams p;
  p.spins = c->spins;
  p.samples = c->d_sd;
  p.blocks = c->d_conv_blocks;
  p.xyz = xyz;
  p.xyz_off = xyz_off;
  p.G = c->G;
  p.Wp = c->Wp;
  p.W = c->W;
  p.fdG_m = c->fdG_m;
  p.fdG_s = c->fdG_s;
  p.seed_lo = c->seed_lo;
  p.seed_hi = c->seed_hi;
  return p;
}

// One sweep of the block table range [b0, b1) (all of it by default): the
// even half-sweep, then the odd one.  With `energy`, both launches also leave
// the per-block energy partials of the new state.
hsg_status half_sweeps(hsg_ctx* c, bool hb, int sweep_offset, bool energy = false, int b0 = 0,
                       int b1 = -1) {
  if (b1 < 0) b1 = c->n_sweep_blocks;
  if (!hb && c->use_staged) {
    int off = 0;
    const size_t smem = staged_smem(c->fmt, c->GPT, energy, c->Lh_max, &off);
    for (int parity = 0; parity < 2; ++parity) {
      SweepParams p = sweep_params(c, parity, sweep_offset);
      p.blk_base = b0;
      p.n_launch = b1 - b0;
      p.reverse = parity;
      p.stage_off = off;
      HSG_CUDA(c, launch_staged_half(c->fmt, c->j16, energy, p, b1 - b0, smem, c->stream));
    }
    return HSG_OK;
  }
  if (!hb && c->use_wave) {
    // both half-sweeps in one launch; the ticket order of the block range is
    // the concatenation of its passes' orders
    WaveParams w;
    w.sw = sweep_params(c, 0, sweep_offset);
    int off = 0;
    size_t smem = c->staged_possible ? staged_smem(c->fmt, c->GPT, energy, c->Lh_max, &off)
                                     : (energy ? sizeof(float) * (SWEEP_BS / 32) * c->GPT * c->VEC : 0);
    w.sw.stage_off = off;
    w.order = c->d_wave_order;
    w.deps = c->d_wave_deps;
    w.flags = c->d_wave_flags;
    w.state = c->d_wave_state;
    w.err = c->d_bar + 5;
    w.timeout_ns = (unsigned long long)std::max(1, c->opt.barrier_timeout_ms) * 1000000ull;
    w.t0 = 2 * b0;
    w.n_tickets = 2 * (b1 - b0);
    w.never = (int)c->max_sweep_blocks;
    w.inject_block = -1;
    // fault injection (tests only; not inside a step graph, which every replay would repeat):
    // the first odd block of the range also waits for a flag no block sets
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    HSG_CUDA(c, cudaStreamIsCapturing(c->stream, &cap));
    if (c->inject_fault && cap == cudaStreamCaptureStatusNone) {
      w.inject_block = b0;
      c->inject_fault = false;
    }
    HSG_CUDA(c, launch_wave(c->fmt, c->j16, energy, c->staged_possible, w, smem, c->stream));
    return HSG_OK;
  }
  for (int parity = 0; parity < 2; ++parity) {
    SweepParams p = sweep_params(c, parity, sweep_offset);
    p.blk_base = b0;
    p.n_launch = b1 - b0;
    // Consecutive launches walk the planes in opposite directions (the blocks
    // of a launch are independent, so the order changes no result): each
    // launch starts on the planes whose spins the previous one left in L2.
    // Packed formats: the decode launch runs forward, the sweep backward.
    p.reverse = c->dec_once ? 1 : parity;
    // packed formats: decode the other parity once for the six neighbour loads
    if (c->dec_once) HSG_CUDA(c, launch_decode_parity(c->fmt, p, 1 - parity, b1 - b0, c->stream));
    HSG_CUDA(c, launch_half_sweep(c->fmt, hb, c->j16, c->opt.fast_math != 0, energy, c->dec_once, p,
                                  b1 - b0, c->stream));
  }
  return HSG_OK;
}

hsg_status enqueue_energy(hsg_ctx* c) {
  EnergyParams p = energy_params(c);
  HSG_CUDA(c, launch_energy(c->fmt, c->j16, p, c->stream));
  return HSG_OK;
}

// Plan of the fused over-relaxation sweep (at first use).  Per sample, the rows
// of y a block holds: the whole plane (rows wrap in the slot) or bands of ny
// rows (the last band may be shorter) with one halo row of even sites and two
// of odd sites on each side.  A step updates R0 = ny + 2 rows of even sites and
// ny rows of odd sites with FUSED_THREADS threads, so the band height is the one
// that fits shared memory and wastes the fewest thread slots on halo rows and
// idle threads (at L = 128: 7 rows, 1024 sites, exactly 2 per thread).  The
// work items are columns (sample, band, chunk group; chunk groups adjacent, so
// blocks that run together share couplings and halo rows in L2) over all
// planes, in whole rounds of the grid; the columns left over are cut into z
// segments so that the last round also fills the grid.  Leaves use_fused off
// unless everything fits.
hsg_status plan_fused(hsg_ctx* c) {
  if (!c->fused_possible || c->d_fused_items) return HSG_OK;
  const int CH = c->VEC * c->ELEM, PL = c->PL;
  int optin = 0, n_sm = 0;
  HSG_CUDA(c, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
  HSG_CUDA(c, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device));
  const long long budget = (long long)optin - FUSED_SMEM_HEAD;
  long long slot1 = 0, slot0 = 0;
  std::vector<int> ny(c->ns, 0);
  for (int s = 0; s < c->ns; ++s) {
    const int L = c->L[s], Lh = L / 2;
    auto fits = [&](int rows1, int rows0) {
      const long long a = std::max(slot1, (long long)PL * rows1 * Lh * CH);
      const long long b = std::max(slot0, (long long)PL * rows0 * Lh * CH);
      return FUSED_ODD_SLOTS * a + FUSED_EVEN_SLOTS * b <= budget;
    };
    // useful site updates per thread slot of a step
    auto score = [&](int n, bool full) {
      const long long sites = full ? 2ll * L * Lh : (long long)(2 * n + 2) * Lh;
      const long long passes = (sites + FUSED_THREADS - 1) / FUSED_THREADS;
      if (passes > FUSED_SITES_PER_THREAD) return -1.0;
      return (double)(2ll * n * Lh) / (double)(passes * FUSED_THREADS);
    };
    int best = 0;
    double best_score = 0.0;
    if (fits(L, L)) {
      best_score = score(L, true);
      if (best_score > 0.0) best = L;
    }
    for (int n = 2; n <= L - 4; ++n) {
      const double sc = score(n, false);
      if (sc > best_score + 1e-9 && fits(n + 4, n + 2)) {
        best = n;
        best_score = sc;
      }
    }
    if (!best) {
      c->fused_possible = false;
      return HSG_OK;
    }
    ny[s] = best;
    const int r1 = best == L ? L : best + 4, r0 = best == L ? L : best + 2;
    slot1 = std::max(slot1, (long long)PL * r1 * Lh * CH);
    slot0 = std::max(slot0, (long long)PL * r0 * Lh * CH);
  }
  const size_t smem = FUSED_SMEM_HEAD + FUSED_ODD_SLOTS * slot1 + FUSED_EVEN_SLOTS * slot0;
  int per_sm = 0;
  HSG_CUDA(c, prepare_fused(c->fmt, c->j16, smem, &per_sm));
  if (per_sm < 1) {
    c->fused_possible = false;
    return HSG_OK;
  }
  const int P = n_sm * per_sm;
  // columns: (sample, chunk group, y0 | rows << 16, L); the last band of a sample may be shorter
  std::vector<int4> cols;
  for (int s = 0; s < c->ns; ++s)
    for (int y0 = 0; y0 < c->L[s]; y0 += ny[s]) {
      const int rows = std::min(ny[s], c->L[s] - y0);
      for (int g = 0; g < c->G; ++g) cols.push_back(make_int4(s, g, y0 | (rows << 16), c->L[s]));
    }
  const int C = (int)cols.size();
  const int full = (C / P) * P, rem = C - full;
  std::vector<int4> items;
  for (int i = 0; i < full; ++i) items.push_back(make_int4(cols[i].x, cols[i].y, cols[i].z, cols[i].w << 16));
  if (rem) {
    int S = std::max(1, P / rem);
    for (int i = full; i < C; ++i) S = std::min(S, std::max(1, cols[i].w / 4));
    for (int k = 0; k < S; ++k)
      for (int i = full; i < C; ++i) {
        const int L = cols[i].w, za = k * L / S, zb = (k + 1) * L / S;
        items.push_back(make_int4(cols[i].x, cols[i].y, cols[i].z, za | (zb << 16)));
      }
  }
  HSG_TRY(dev_alloc(c, &c->spins2, c->spin_bytes));
  HSG_TRY(dev_alloc(c, &c->d_fused_items, sizeof(int4) * items.size()));
  HSG_CUDA(c, cudaMemcpy(c->d_fused_items, items.data(), sizeof(int4) * items.size(),
                         cudaMemcpyHostToDevice));
  c->n_fused_items = (int)items.size();
  c->fused_grid = std::min(P, c->n_fused_items);
  c->fused_smem = smem;
  c->fused_slot1 = (uint32_t)slot1;
  c->fused_slot0 = (uint32_t)slot0;
  c->fused_ny = ny;
  return HSG_OK;
}

// `pairs` pairs of fused over-relaxation sweeps: spins -> spins2 -> spins.
hsg_status fused_sweep_pairs(hsg_ctx* c, int pairs) {
  FusedParams p;
  p.rec = c->rec;
  p.samples = c->d_sd;
  p.items = c->d_fused_items;
  p.active = c->d_active;
  p.n_items = c->n_fused_items;
  p.slot1 = c->fused_slot1;
  p.slot0 = c->fused_slot0;
  p.err = c->d_bar + 4;
  p.timeout_ns = (unsigned long long)std::max(1, c->opt.barrier_timeout_ms) * 1000000ull;
  for (int k = 0; k < pairs; ++k) {
    p.src = c->spins;
    p.dst = c->spins2;
    HSG_CUDA(c, launch_fused(c->fmt, c->j16, p, c->fused_grid, c->fused_smem, c->stream));
    p.src = c->spins2;
    p.dst = c->spins;
    HSG_CUDA(c, launch_fused(c->fmt, c->j16, p, c->fused_grid, c->fused_smem, c->stream));
  }
  return HSG_OK;
}

// n OR sweeps outside a step: fused pairs where in use, the rest per half-sweep.
hsg_status or_sweeps(hsg_ctx* c, int n, int sweep_offset) {
  int k = 0;
  if (c->use_fused && n >= 2) {
    HSG_TRY(fused_sweep_pairs(c, n / 2));
    k = 2 * (n / 2);
  }
  for (; k < n; ++k) HSG_TRY(half_sweeps(c, false, sweep_offset + k));
  return HSG_OK;
}

// A step: n_hb HB sweeps, n_or OR sweeps (the last one also produces the
// energy partials of the final state), the energy sums and one PT pass.  The
// sweeps run pass by pass; systems are independent and every random number is
// keyed by (site, system, sweep), so the order of the passes changes nothing.
hsg_status enqueue_step(hsg_ctx* c) {
  const int nhb = c->opt.n_hb_per_step, nor = c->opt.n_or_per_step;
  const int np = (int)c->pass_bound.size() - 1;
  for (int ps = 0; ps < np; ++ps) {
    const int b0 = c->pass_bound[ps], b1 = c->pass_bound[ps + 1];
    for (int k = 0; k < nhb; ++k) HSG_TRY(half_sweeps(c, true, k, false, b0, b1));
    int k = 0;
    if (c->use_fused && np == 1) {
      // pairs of fused sweeps, leaving the last sweep (which also sums the
      // energies) to the per-half-sweep kernel
      const int pairs = (nor - 1) / 2;
      HSG_TRY(fused_sweep_pairs(c, pairs));
      k = 2 * pairs;
    }
    for (; k < nor; ++k) HSG_TRY(half_sweeps(c, false, nhb + k, k == nor - 1, b0, b1));
  }
  if (nor > 0) {
    HSG_CUDA(c, launch_energy_final_pt(energy_params(c), pt_params(c, nhb + nor, 1), c->stream));
  } else {
    HSG_TRY(enqueue_energy(c));
    HSG_CUDA(c, launch_pt(pt_params(c, nhb + nor, 1), c->stream));
  }
  return HSG_OK;
}

// A bounded device wait that ran out (persistent schedule, staged measurement)
// after the stream has been synchronised.
hsg_status poll_device_error(hsg_ctx* c) {
  unsigned int err[5] = {0u, 0u, 0u, 0u, 0u};
  HSG_CUDA(c, cudaMemcpy(err, c->d_bar + 2, sizeof(err), cudaMemcpyDeviceToHost));
  if (err[4]) return fail(c, HSG_ESTATE, "a device bounds check of a sweep kernel failed (HSG_CHECK build)");
  if (err[0]) return fail(c, HSG_ETIMEOUT, "a grid barrier wait of the persistent step kernel timed out");
  if (err[1]) return fail(c, HSG_ETIMEOUT, "a wait for a staged spin copy of a measurement kernel timed out");
  if (err[2]) return fail(c, HSG_ETIMEOUT, "a wait for a staged plane copy of the fused sweep kernel timed out");
  if (err[3]) return fail(c, HSG_ETIMEOUT, "a wait of the wave sweep kernel for its even blocks timed out");
  return HSG_OK;
}

PersistParams persist_params(hsg_ctx* c, int n_steps) {
  PersistParams P;
  P.sw = sweep_params(c, 0, 0);
  P.en = energy_params(c);
  P.pt = pt_params(c, 0, 1);
  P.bar = c->d_bar;
  P.timeout_ns = (unsigned long long)std::max(1, c->opt.barrier_timeout_ms) * 1000000ull;
  P.n_steps = n_steps;
  P.nhb = c->opt.n_hb_per_step;
  P.nor = c->opt.n_or_per_step;
  P.drop_first = c->inject_fault ? 1 : 0;
  P.pass_bound = c->d_pass_bound;
  P.n_passes = (int)c->pass_bound.size() - 1;
  return P;
}

hsg_status ensure_xyz(hsg_ctx* c) {
  if (c->d_xyz) return HSG_OK;
  HSG_TRY(dev_alloc(c, &c->d_xyz, (size_t)c->xyz_floats * sizeof(float)));
  HSG_TRY(dev_alloc(c, &c->d_xyz_off, c->xyz_off.size() * sizeof(long long)));
  HSG_CUDA(c, cudaMemcpy(c->d_xyz_off, c->xyz_off.data(), c->xyz_off.size() * sizeof(long long),
                         cudaMemcpyHostToDevice));
  return HSG_OK;
}

bool finite_all(const float* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// chunks per thread: enough threads to fill the GPU (~152 SMs x 2048); the
// rest of the chunks are walked by each thread, so that the site geometry and
// couplings are computed once per site
int default_gpt(hsg_ctx*, const int* L, int n_samples, int G) {
  long long half_sites = 0;
  for (int s = 0; s < n_samples; ++s) half_sites += (long long)L[s] * L[s] * L[s] / 2;
  const long long gpt = half_sites * G / (152ll * 2048);
  return (int)std::max(1ll, std::min((long long)G, gpt));
}

// Plan of the wave sweep for the block table `blocks` and the passes in
// c->pass_bound.  An odd block covering planes [z0, z1] of its sample and chunk
// group depends on the even blocks of planes z0-1 .. z1+1 (periodic; at most two
// ranges of the table).  Per pass, the even blocks go in the order (sample,
// first site, chunk group) and each odd block is placed `lag` even blocks after
// the last even block it depends on, so every dependency holds an earlier ticket.
hsg_status plan_wave(hsg_ctx* c, const std::vector<int4>& blocks, int lag) {
  if (!c->d_wave_order) {
    HSG_TRY(dev_alloc(c, &c->d_wave_order, sizeof(int) * 2 * c->max_sweep_blocks));
    HSG_TRY(dev_alloc(c, &c->d_wave_deps, sizeof(int4) * c->max_sweep_blocks));
    // (one more flag than blocks: the one fault injection waits for, never set)
    HSG_TRY(dev_alloc(c, &c->d_wave_flags, sizeof(unsigned int) * (c->max_sweep_blocks + 1)));
    HSG_TRY(dev_alloc(c, &c->d_wave_state, sizeof(unsigned int) * 4));
    HSG_CUDA(c, cudaMemset(c->d_wave_flags, 0, sizeof(unsigned int) * (c->max_sweep_blocks + 1)));
    HSG_CUDA(c, cudaMemset(c->d_wave_state, 0, sizeof(unsigned int) * 4));
  }
  if (lag <= 0) {
    int per_sm = 0, n_sm = 0, off = 0;
    const size_t smem = c->staged_possible ? staged_smem(c->fmt, c->GPT, false, c->Lh_max, &off) : 0;
    HSG_CUDA(c, wave_occupancy(c->fmt, c->j16, c->staged_possible, smem, &per_sm));
    HSG_CUDA(c, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device));
    lag = std::max(1, n_sm * per_sm / 2);
  }
  const int nb = (int)blocks.size();
  std::vector<int4> deps(nb, make_int4(0, 0, 0, 0));
  std::vector<int> order(2 * (size_t)nb);
  for (size_t ps = 0; ps + 1 < c->pass_bound.size(); ++ps) {
    const int b0 = c->pass_bound[ps], b1 = c->pass_bound[ps + 1];
    // even blocks sample by sample, plane by plane, and within a run of sites
    // all chunk groups: the blocks in flight then cover few planes (with all
    // their systems), which keeps what the odd blocks re-read small enough for L2
    std::vector<int> epos_order;
    for (int b = b0; b < b1; ++b) epos_order.push_back(b);
    std::stable_sort(epos_order.begin(), epos_order.end(), [&](int a, int b) {
      if (blocks[a].x != blocks[b].x) return blocks[a].x < blocks[b].x;
      if (blocks[a].z != blocks[b].z) return blocks[a].z < blocks[b].z;
      return blocks[a].y < blocks[b].y;
    });
    std::vector<int> epos(b1 - b0);
    for (int q = 0; q < b1 - b0; ++q) epos[epos_order[q] - b0] = q;
    std::vector<std::pair<long long, int>> keyed;   // (position key, ticket code)
    keyed.reserve(2 * (size_t)(b1 - b0));
    for (int b = b0; b < b1; ++b) {
      const int4 k = blocks[b];
      const SampleDev& d = c->sd[k.x];
      const int L = d.L;
      const long long P = (long long)L * d.Lh, half = d.N / 2;   // half-sites per plane, per parity
      const int per_g = (int)((half + SWEEP_BS - 1) / SWEEP_BS);
      const int e_first = d.blk0 + k.y * per_g;
      const long long h_end = std::min<long long>((long long)k.z + SWEEP_BS, half);
      const int z0 = (int)(k.z / P), z1 = (int)((h_end - 1) / P);
      // even blocks of planes [p0, p1] (no wrap): [first, last + 1)
      auto range = [&](int p0, int p1) {
        return std::make_pair(e_first + (int)(p0 * P / SWEEP_BS),
                              e_first + (int)(((p1 + 1) * P - 1) / SWEEP_BS) + 1);
      };
      int4 dep;
      if (z1 - z0 + 3 >= L) {
        dep = make_int4(e_first, e_first + per_g, 0, 0);
      } else if (z0 == 0) {
        const auto r1 = range(0, z1 + 1), r2 = range(L - 1, L - 1);
        dep = make_int4(r1.first, r1.second, r2.first, r2.second);
      } else if (z1 == L - 1) {
        const auto r1 = range(z0 - 1, L - 1), r2 = range(0, 0);
        dep = make_int4(r1.first, r1.second, r2.first, r2.second);
      } else {
        const auto r = range(z0 - 1, z1 + 1);
        dep = make_int4(r.first, r.second, 0, 0);
      }
      deps[b] = dep;
      if (dep.x < b0 || dep.y > b1 || dep.x >= dep.y || (dep.w > dep.z && (dep.z < b0 || dep.w > b1)))
        return fail(c, HSG_ESTATE, "wave sweep plan: dependency outside the pass");
      int last = 0;   // the latest position among the even blocks it depends on
      for (int e = dep.x; e < dep.y; ++e) last = std::max(last, epos[e - b0]);
      for (int e = dep.z; e < dep.w; ++e) last = std::max(last, epos[e - b0]);
      keyed.push_back({2ll * epos[b - b0], b << 1});
      keyed.push_back({2ll * ((long long)last + lag) + 1, (b << 1) | 1});
    }
    std::stable_sort(keyed.begin(), keyed.end(),
                     [](const std::pair<long long, int>& a, const std::pair<long long, int>& b) {
                       return a.first < b.first;
                     });
    for (size_t i = 0; i < keyed.size(); ++i) order[2 * (size_t)b0 + i] = keyed[i].second;
    // check before any launch: each dependency is an even block of the same
    // sample and chunk group inside this pass, with an earlier ticket
    std::vector<int> ticket(b1 - b0, -1);
    for (size_t i = 0; i < keyed.size(); ++i)
      if ((keyed[i].second & 1) == 0) ticket[(keyed[i].second >> 1) - b0] = (int)i;
    for (size_t i = 0; i < keyed.size(); ++i) {
      if ((keyed[i].second & 1) == 0) continue;
      const int b = keyed[i].second >> 1;
      const int4 k = blocks[b], dep = deps[b];
      for (const auto& r : {std::make_pair(dep.x, dep.y), std::make_pair(dep.z, dep.w)})
        for (int e = r.first; e < r.second; ++e)
          if (e < b0 || e >= b1 || blocks[e].x != k.x || blocks[e].y != k.y || ticket[e - b0] >= (int)i)
            return fail(c, HSG_ESTATE, "wave sweep plan: bad dependency");
    }
  }
  HSG_CUDA(c, cudaMemcpyAsync(c->d_wave_order, order.data(), sizeof(int) * order.size(),
                              cudaMemcpyHostToDevice, c->stream));
  HSG_CUDA(c, cudaMemcpyAsync(c->d_wave_deps, deps.data(), sizeof(int4) * deps.size(),
                              cudaMemcpyHostToDevice, c->stream));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  c->wave_lag = lag;
  return HSG_OK;
}

// Build the sweep block table for `gpt` chunks per thread, cut it into passes
// whose footprint (spins of their chunk groups plus the records of their
// samples) stays within `pass_bytes` (0: one pass; a pass holds at least one
// chunk group), and set up the chosen step schedule (drops a captured graph:
// its parameters change).
hsg_status configure_schedule(hsg_ctx* c, int variant, int gpt, long long pass_bytes, int sweep,
                              int lag) {
  gpt = std::max(1, std::min(c->G, gpt));
  const int n_gg = (c->G + gpt - 1) / gpt;
  const long long site_chunk_bytes = (long long)c->PL * c->VEC * c->ELEM;
  const long long site_rec_bytes = 12ll * (c->j16 ? 2 : 4);
  std::vector<int4> blocks;
  std::vector<int> bounds{0};
  long long used = 0;
  int last_sample = -1;
  int max_rows = 1;
  for (int s = 0; s < c->ns; ++s) {
    SampleDev& d = c->sd[s];
    d.blk0 = (int)blocks.size();
    for (int gg = 0; gg < n_gg; ++gg) {
      const int chunks = std::min(gpt, c->G - gg * gpt);
      long long add = (long long)d.N * chunks * site_chunk_bytes;
      if (s != last_sample) add += (long long)d.N * site_rec_bytes;
      if (pass_bytes > 0 && (int)blocks.size() > bounds.back() && used + add > pass_bytes) {
        bounds.push_back((int)blocks.size());
        used = 0;
        add = (long long)d.N * (chunks * site_chunk_bytes + site_rec_bytes);
      }
      used += add;
      last_sample = s;
      for (int h0 = 0; h0 < d.N / 2; h0 += SWEEP_BS) blocks.push_back(make_int4(s, gg, h0, 0));
    }
    d.blk1 = (int)blocks.size();
    max_rows = std::max(max_rows, d.blk1 - d.blk0);
  }
  bounds.push_back((int)blocks.size());
  if ((long long)blocks.size() > c->max_sweep_blocks) return fail(c, HSG_ESTATE, "sweep table overflow");
  if ((int)bounds.size() - 1 > c->max_passes) return fail(c, HSG_ESTATE, "pass table overflow");
  c->GPT = gpt;
  c->n_sweep_blocks = (int)blocks.size();
  c->pass_bound = bounds;
  c->pass_bytes = pass_bytes;
  HSG_CUDA(c, cudaMemcpyAsync(c->d_pass_bound, bounds.data(), sizeof(int) * bounds.size(),
                              cudaMemcpyHostToDevice, c->stream));
  // energy sums: about 16 block rows per first-level unit, at most MAX_E_SPLITS
  c->e_splits = std::min(MAX_E_SPLITS, std::max(1, max_rows / 16));
  HSG_CUDA(c, cudaMemcpyAsync(c->d_sweep_blocks, blocks.data(), sizeof(int4) * blocks.size(),
                              cudaMemcpyHostToDevice, c->stream));
  HSG_CUDA(c, cudaMemcpyAsync(c->d_sd, c->sd.data(), sizeof(SampleDev) * c->ns,
                              cudaMemcpyHostToDevice, c->stream));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  if (c->graph) {
    cudaGraphDestroy(c->graph);
    c->graph = nullptr;
  }
  c->variant = variant;
  // the fused over-relaxation sweep serves the two-pass schedule in one pass,
  // the wave sweep the two-pass schedule with any passes
  c->use_fused = false;
  c->use_wave = false;
  c->use_staged = sweep == HSG_SWEEP_STAGED && variant == HSG_VARIANT_TWO_PASS && c->staged_possible;
  if (sweep == HSG_SWEEP_FUSED && variant == HSG_VARIANT_TWO_PASS && bounds.size() == 2) {
    HSG_TRY(plan_fused(c));
    c->use_fused = c->fused_possible;
  }
  if (sweep == HSG_SWEEP_WAVE && variant == HSG_VARIANT_TWO_PASS && c->wave_possible) {
    HSG_TRY(plan_wave(c, blocks, lag));
    c->use_wave = true;
  }
  if (variant == HSG_VARIANT_PERSISTENT) {
    c->persist_smem = sizeof(float) * (SWEEP_BS / 32) * c->GPT * c->VEC;
    int max_grid = 0;
    HSG_CUDA(c, max_persistent_grid(c->fmt, c->j16, c->opt.fast_math != 0, c->persist_smem, &max_grid));
    if (max_grid < 2) return fail(c, HSG_ECUDA, "persistent kernel does not fit on the device");
    const int wgs = (c->Wp + 31) / 32;
    long long need = std::max<long long>(c->n_sweep_blocks, (long long)c->e_splits * wgs * c->ns);
    need = std::max<long long>(need, ((long long)c->ns * c->Wp + SWEEP_BS - 1) / SWEEP_BS);
    c->persist_grid = (int)std::max(2ll, std::min<long long>(max_grid, need));
  }
  return HSG_OK;
}

// n_steps steps with the configured schedule (graph captured on first use).
hsg_status run_steps(hsg_ctx* c, int n_steps) {
  if (c->variant == HSG_VARIANT_PERSISTENT) {
    HSG_CUDA(c, cudaMemsetAsync(c->d_bar, 0, sizeof(unsigned int), c->stream));
    PersistParams P = persist_params(c, n_steps);
    c->inject_fault = false;
    HSG_CUDA(c, launch_persistent(c->fmt, c->j16, c->opt.fast_math != 0, P, c->persist_grid,
                                  c->persist_smem, c->stream));
    return HSG_OK;
  }
  if (!c->graph_exec) {
    HSG_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    hsg_status st = enqueue_step(c);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (st != HSG_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    HSG_CUDA(c, e);
    c->graph = g;
    HSG_CUDA(c, cudaGraphInstantiate(&c->graph_exec, c->graph, 0));
  }
  for (int k = 0; k < n_steps; ++k) HSG_CUDA(c, cudaGraphLaunch(c->graph_exec, c->stream));
  return HSG_OK;
}

// The device arrays that, with the spins, make up the state of the Markov chain
// and its statistics (what a checkpoint holds and the autotuner restores).
std::vector<std::pair<void*, size_t>> chain_regions(hsg_ctx* c) {
  const size_t n_perm = (size_t)c->ns * c->R_O * c->R_T;
  const size_t n_acc = (size_t)c->ns * c->R_O * std::max(1, c->R_T - 1);
  return {{c->d_perm, sizeof(int) * n_perm},
          {c->d_beta, sizeof(float) * c->ns * (size_t)c->Wp},
          {c->d_E, sizeof(double) * c->ns * (size_t)c->Wp},
          {c->d_acc, sizeof(unsigned long long) * n_acc},
          {c->d_counters, sizeof(unsigned long long) * 2 * c->ns},
          {c->d_moved, sizeof(unsigned long long) * n_perm},
          {c->d_tstate, sizeof(unsigned char) * n_perm},
          {c->d_tunnel, sizeof(unsigned int) * n_perm}};
}

size_t chain_state_bytes(hsg_ctx* c) {
  size_t n = 0;
  for (auto& r : chain_regions(c)) n += r.second;
  return n;
}

// Copy the chain-state regions to or from consecutive host bytes (stream-ordered).
hsg_status copy_chain_state(hsg_ctx* c, unsigned char* host, bool to_host) {
  size_t off = 0;
  for (auto& r : chain_regions(c)) {
    if (to_host)
      HSG_CUDA(c, cudaMemcpyAsync(host + off, r.first, r.second, cudaMemcpyDeviceToHost, c->stream));
    else
      HSG_CUDA(c, cudaMemcpyAsync(r.first, host + off, r.second, cudaMemcpyHostToDevice, c->stream));
    off += r.second;
  }
  return HSG_OK;
}

// Autotuner: the schedules, sweep kernels and chunks-per-thread settings
// compute identical results, so they are timed on the live context and the
// fastest is kept (by a margin of 1%); the state is saved before and restored after, so the
// Markov chain is untouched.  Each candidate runs one warm-up step, then
// TUNE_REPS timings of 2 steps each; the median decides (a single timing let
// noise pick between close candidates).  Results are cached per problem shape
// for the life of the process.
struct TuneChoice {
  int variant, gpt;
  long long pass_bytes;
  int sweep, lag;
};
constexpr int TUNE_REPS = 5;
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune_cache;

std::string tune_key(hsg_ctx* c) {
  std::string k = std::to_string(c->fmt) + "/" + std::to_string(c->j16) + "/" +
                  std::to_string(c->opt.fast_math) + "/" + std::to_string(c->W) + "/" +
                  std::to_string(c->opt.n_hb_per_step) + "/" + std::to_string(c->opt.n_or_per_step) +
                  "/" + std::to_string(c->opt.pass_bytes) + "/" +
                  std::to_string(c->opt.chunks_per_thread) + "/" +
                  std::to_string(c->opt.sweep_kernel) + "/" + std::to_string(c->opt.wave_lag) + "/L";
  for (int L : c->L) k += std::to_string(L) + ",";
  return k;
}

hsg_status autotune(hsg_ctx* c) {
  c->tune_pending = false;
  const std::string key = tune_key(c);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end())
      return configure_schedule(c, it->second.variant, it->second.gpt, it->second.pass_bytes,
                                it->second.sweep, it->second.lag);
  }
  // save the state the trial steps will change
  void* spins_copy = nullptr;
  HSG_CUDA(c, cudaMalloc(&spins_copy, c->spin_bytes));
  std::vector<unsigned char> saved(chain_state_bytes(c));
  cudaStream_t st = c->stream;
  const bool e_valid = c->e_valid;
  HSG_CUDA(c, cudaMemcpyAsync(spins_copy, c->spins, c->spin_bytes, cudaMemcpyDeviceToDevice, st));
  HSG_TRY(copy_chain_state(c, saved.data(), true));
  HSG_CUDA(c, cudaStreamSynchronize(st));

  std::vector<int> gpts;
  for (int g : {c->G, (c->G + 1) / 2, (c->G + 3) / 4, 2, 1, c->GPT})
    if (g >= 1 && g <= c->G && std::find(gpts.begin(), gpts.end(), g) == gpts.end()) gpts.push_back(g);
  if (c->opt.chunks_per_thread > 0) gpts.assign(1, c->GPT);
  // over-relaxation sweep kernels (with the wave sweep's lags) to try
  std::vector<std::pair<int, int>> sweeps;
  const int sk = c->opt.sweep_kernel;
  if (sk == HSG_SWEEP_AUTO || sk == HSG_SWEEP_HALF) sweeps.push_back({HSG_SWEEP_HALF, 0});
  if ((sk == HSG_SWEEP_AUTO || sk == HSG_SWEEP_FUSED) && c->fused_possible && c->opt.n_or_per_step >= 3)
    sweeps.push_back({HSG_SWEEP_FUSED, 0});
  // the wave sweep only on request (slower than two half-sweep launches on every
  // shape measured): at the requested lag, or at half and twice the default
  if (sk == HSG_SWEEP_WAVE && c->wave_possible) {
    if (c->opt.wave_lag > 0) {
      sweeps.push_back({HSG_SWEEP_WAVE, c->opt.wave_lag});
    } else {
      int per_sm = 0, n_sm = 0, off = 0;
      const size_t smem = c->staged_possible ? staged_smem(c->fmt, c->GPT, false, c->Lh_max, &off) : 0;
      HSG_CUDA(c, wave_occupancy(c->fmt, c->j16, c->staged_possible, smem, &per_sm));
      HSG_CUDA(c, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device));
      const int resident = std::max(4, n_sm * per_sm);
      for (int lag : {resident / 4, resident}) sweeps.push_back({HSG_SWEEP_WAVE, lag});
    }
  }
  if ((sk == HSG_SWEEP_AUTO || sk == HSG_SWEEP_STAGED) && c->staged_possible)
    sweeps.push_back({HSG_SWEEP_STAGED, 0});
  if (sweeps.empty()) sweeps.push_back({HSG_SWEEP_HALF, 0});
  cudaEvent_t e0, e1;
  HSG_CUDA(c, cudaEventCreate(&e0));
  HSG_CUDA(c, cudaEventCreate(&e1));
  // pass footprints: one pass, and passes that fit the L2 cache (then every
  // sweep of a pass after the first reads its spins and records from L2)
  std::vector<long long> budgets;
  if (c->opt.pass_bytes > 0) {
    budgets.push_back(c->opt.pass_bytes);
  } else {
    int l2 = 0;
    HSG_CUDA(c, cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device));
    budgets.push_back(0);
    if (l2 > 0 && (long long)c->spin_bytes + (long long)c->rec_bytes > l2 / 2) {
      budgets.push_back((long long)l2 * 3 / 4);
      budgets.push_back((long long)l2 / 2);
    }
  }
  float best = 1e30f;
  TuneChoice bestc{HSG_VARIANT_TWO_PASS, c->GPT, budgets[0], sweeps[0].first, sweeps[0].second};
  for (long long pb : budgets) {
    for (int v : {HSG_VARIANT_TWO_PASS, HSG_VARIANT_PERSISTENT}) {
      for (const auto& sw : sweeps) {
        // the fused sweep runs in the two-pass schedule with one pass only, the
        // wave sweep in the two-pass schedule; the persistent schedule has its own
        if (sw.first != HSG_SWEEP_HALF && v != HSG_VARIANT_TWO_PASS) continue;
        if (sw.first == HSG_SWEEP_FUSED && pb != 0) continue;
        for (int g : gpts) {
          HSG_TRY(configure_schedule(c, v, g, pb, sw.first, sw.second));
          if (sw.first == HSG_SWEEP_FUSED && !c->use_fused) continue;
          HSG_TRY(run_steps(c, 1));
          float t[TUNE_REPS];
          for (int r = 0; r < TUNE_REPS; ++r) {
            HSG_CUDA(c, cudaEventRecord(e0, st));
            HSG_TRY(run_steps(c, 2));
            HSG_CUDA(c, cudaEventRecord(e1, st));
            HSG_CUDA(c, cudaEventSynchronize(e1));
            HSG_CUDA(c, cudaEventElapsedTime(&t[r], e0, e1));
          }
          HSG_TRY(poll_device_error(c));
          std::sort(t, t + TUNE_REPS);
          const float ms = t[TUNE_REPS / 2];
          // a candidate replaces the current choice only when it is at least
          // 1% faster, so that timing noise between near-equal candidates does
          // not decide (candidates are tried simplest first)
          if (ms < best * 0.99f) {
            best = ms;
            bestc = TuneChoice{v, g, pb, sw.first, sw.second};
          }
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // restore
  HSG_CUDA(c, cudaMemcpyAsync(c->spins, spins_copy, c->spin_bytes, cudaMemcpyDeviceToDevice, st));
  HSG_TRY(copy_chain_state(c, saved.data(), false));
  HSG_CUDA(c, cudaStreamSynchronize(st));
  HSG_CUDA(c, cudaFree(spins_copy));
  c->e_valid = e_valid;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = bestc;
  }
  return configure_schedule(c, bestc.variant, bestc.gpt, bestc.pass_bytes, bestc.sweep, bestc.lag);
}

hsg_status create_impl(hsg_ctx** out, int n_samples, const int* L, const double* temps,
                       int n_temps, int n_replicas, const float* const* J,
                       const float* const* H, uint64_t seed, const hsg_options* optp) {
  if (!out) return bad_arg(nullptr, "out is NULL");
  *out = nullptr;
  hsg_options opt;
  hsg_default_options(&opt);
  if (optp) opt = *optp;
  // samples index a grid dimension of the energy and measurement launches
  if (n_samples < 1 || n_samples > 65535) return bad_arg(nullptr, "n_samples must be in [1, 65535]");
  if (!L || !temps || !J) return bad_arg(nullptr, "L, temps and J must not be NULL");
  if (n_temps < 1 || n_temps > 256) return bad_arg(nullptr, "n_temps must be in [1, 256]");
  if (n_replicas < 1) return bad_arg(nullptr, "n_replicas < 1");
  if (opt.precision < HSG_FP32 || opt.precision > HSG_YX4)
    return bad_arg(nullptr, "unknown precision");
  if (opt.n_hb_per_step < 0 || opt.n_or_per_step < 0)
    return bad_arg(nullptr, "negative sweeps per step");
  if (opt.pass_bytes < 0) return bad_arg(nullptr, "pass_bytes < 0");
  if (opt.variant < HSG_VARIANT_AUTO || opt.variant > HSG_VARIANT_PERSISTENT)
    return bad_arg(nullptr, "unknown variant");
  if (opt.chunks_per_thread < 0) return bad_arg(nullptr, "chunks_per_thread < 0");
  if (opt.sweep_kernel < HSG_SWEEP_AUTO || opt.sweep_kernel > HSG_SWEEP_STAGED)
    return bad_arg(nullptr, "unknown sweep_kernel");
  if (opt.wave_lag < 0) return bad_arg(nullptr, "wave_lag < 0");
  if (opt.inject_alloc_fault < 0) return bad_arg(nullptr, "inject_alloc_fault < 0");
  const int W = n_temps * n_replicas;
  if (W > 1024) return bad_arg(nullptr, "n_temps * n_replicas must be <= 1024");
  const int Wp = (W + 7) / 8 * 8;
  const int fmt = opt.precision;
  const int VEC = fmt_vec(fmt), G = Wp / VEC;
  for (int s = 0; s < n_samples; ++s) {
    if (L[s] < 4 || (L[s] & 1) || L[s] > 512)
      return bad_arg(nullptr, "L must be even and in [4, 512]");
    const long long N = (long long)L[s] * L[s] * L[s];
    if (N * G >= (1ll << 31)) return bad_arg(nullptr, "lattice too large for the system count");
    if (!J[s]) return bad_arg(nullptr, "J[s] is NULL");
    if (!finite_all(J[s], (size_t)N * 3)) return bad_arg(nullptr, "J has a non-finite value");
    if (H && H[s] && !finite_all(H[s], (size_t)N * 3))
      return bad_arg(nullptr, "H has a non-finite value");
    for (int t = 0; t < n_temps; ++t) {
      const double T = temps[(size_t)s * n_temps + t];
      if (!std::isfinite(T) || T <= 0.0) return bad_arg(nullptr, "temperatures must be positive");
      if (t > 0 && !(T > temps[(size_t)s * n_temps + t - 1]))
        return bad_arg(nullptr, "temperatures must be strictly increasing");
    }
  }

  hsg_ctx* c = new hsg_ctx();
  c->opt = opt;
  c->alloc_fail_at = opt.inject_alloc_fault;
  c->device = opt.device;
  c->fmt = fmt;
  c->VEC = VEC;
  c->PL = fmt_planes(fmt);
  c->ELEM = fmt_elem(fmt);
  c->j16 = opt.j_fp16 != 0;
  c->ns = n_samples;
  c->R_T = n_temps;
  c->R_O = n_replicas;
  c->W = W;
  c->Wp = Wp;
  c->G = G;
  c->seed_lo = (uint32_t)(seed & 0xffffffffu);
  c->seed_hi = (uint32_t)(seed >> 32);
  fastdiv((uint32_t)G, &c->fdG_m, &c->fdG_s);
  c->L.assign(L, L + n_samples);

  auto cleanup_fail = [&](hsg_status st) {
    g_create_error = c->msg;
    hsg_destroy(c);
    return st;
  };

  cudaError_t e = cudaSetDevice(opt.device);
  if (e != cudaSuccess) {
    c->msg = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
    return cleanup_fail(HSG_ECUDA);
  }
  if (opt.stream) {
    c->stream = (cudaStream_t)opt.stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      c->msg = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
      return cleanup_fail(HSG_ECUDA);
    }
    c->own_stream = true;
  }

  // layout
  std::vector<int4> conv_blocks;
  long long max_sweep_blocks = 0;
  c->GPT = opt.chunks_per_thread > 0 ? std::min(G, opt.chunks_per_thread)
                                     : default_gpt(c, L, n_samples, G);
  size_t spin_off = 0, rec_off = 0;
  long long xyz = 0;
  for (int s = 0; s < n_samples; ++s) {
    SampleDev d{};
    d.L = L[s];
    d.N = L[s] * L[s] * L[s];
    d.Lh = L[s] / 2;
    fastdiv((uint32_t)d.Lh, &d.fdLh_m, &d.fdLh_s);
    fastdiv((uint32_t)d.L, &d.fdL_m, &d.fdL_s);
    d.spin_off = (long long)spin_off;
    d.plane_stride = (long long)d.N * Wp * c->ELEM;
    d.rec_off = (long long)rec_off;
    d.sys_base = s * Wp;
    max_sweep_blocks += (long long)G * ((d.N / 2 + SWEEP_BS - 1) / SWEEP_BS);
    for (int g = 0; g < G; ++g)
      for (int s0 = 0; s0 < d.N; s0 += 256) conv_blocks.push_back(make_int4(s, g, s0, 0));
    size_t sb = (size_t)c->PL * d.plane_stride;
    spin_off += (sb + 255) / 256 * 256;
    if (fmt_decodes_once(fmt)) {
      d.dec_off = (long long)c->dec_bytes;
      d.dec_plane_stride = (long long)(d.N / 2) * Wp * 4;
      c->dec_bytes += ((size_t)3 * d.dec_plane_stride + 255) / 256 * 256;
    }
    rec_off += (size_t)d.N;
    c->sd.push_back(d);
    c->xyz_off.push_back(xyz);
    xyz += (long long)W * d.N * 3;
    c->total_sites += d.N;
    c->Lmax = std::max(c->Lmax, d.L);
  }
  c->xyz_floats = xyz;
  c->spin_bytes = spin_off;
  c->rec_bytes = rec_off * (c->j16 ? 24 : 48);
  c->max_sweep_blocks = max_sweep_blocks;
  c->max_passes = n_samples * G;
  c->n_conv_blocks = (int)conv_blocks.size();

  // records: six bonds and the field of every storage site
  std::vector<float> recf;
  std::vector<__half> rech;
  if (c->j16) rech.resize(rec_off * 12);
  else recf.resize(rec_off * 12);
  for (int s = 0; s < n_samples; ++s) {
    const SampleDev& d = c->sd[s];
    const int Ls = d.L, Lh = d.Lh;
    const long long half_n = d.N / 2;
    const float* Js = J[s];
    const float* Hs = (H && H[s]) ? H[s] : nullptr;
    for (long long ss = 0; ss < d.N; ++ss) {
      const int par = ss >= half_n ? 1 : 0;
      const long long h = ss - par * half_n;
      const long long r = h / Lh;
      const int hx = (int)(h % Lh);
      const int y = (int)(r % Ls), z = (int)(r / Ls);
      const int x = 2 * hx + ((par + y + z) & 1);
      auto idx = [&](int xx, int yy, int zz) {
        return (long long)((xx + Ls) % Ls) + (long long)Ls * (((yy + Ls) % Ls) + (long long)Ls * ((zz + Ls) % Ls));
      };
      const long long i = idx(x, y, z);
      float v[12];
      v[0] = Js[i * 3 + 0];
      v[1] = Js[idx(x - 1, y, z) * 3 + 0];
      v[2] = Js[i * 3 + 1];
      v[3] = Js[idx(x, y - 1, z) * 3 + 1];
      v[4] = Js[i * 3 + 2];
      v[5] = Js[idx(x, y, z - 1) * 3 + 2];
      v[6] = Hs ? Hs[i * 3 + 0] : 0.0f;
      v[7] = Hs ? Hs[i * 3 + 1] : 0.0f;
      v[8] = Hs ? Hs[i * 3 + 2] : 0.0f;
      v[9] = v[10] = v[11] = 0.0f;
      const size_t o = (size_t)(d.rec_off + ss) * 12;
      for (int k = 0; k < 12; ++k) {
        if (c->j16) rech[o + k] = __float2half_rn(v[k]);
        else recf[o + k] = v[k];
      }
    }
  }

  // device allocations
  hsg_status st;
#define HSG_ALLOC(ptr, bytes)                   \
  st = dev_alloc(c, &(ptr), (bytes));           \
  if (st != HSG_OK) return cleanup_fail(st);
  HSG_ALLOC(c->spins, c->spin_bytes);
  c->dec_once = fmt_decodes_once(fmt);
  if (c->dec_once) {
    HSG_ALLOC(c->dec, c->dec_bytes);
  }
  HSG_ALLOC(c->rec, c->rec_bytes);
  HSG_ALLOC(c->d_sd, sizeof(SampleDev) * n_samples);
  HSG_ALLOC(c->d_sweep_blocks, sizeof(int4) * max_sweep_blocks);
  HSG_ALLOC(c->d_pass_bound, sizeof(int) * (c->max_passes + 1));
  HSG_ALLOC(c->d_conv_blocks, sizeof(int4) * conv_blocks.size());
  HSG_ALLOC(c->d_epart, sizeof(double) * 2 * max_sweep_blocks * Wp);
  HSG_ALLOC(c->d_epart2, sizeof(double) * n_samples * MAX_E_SPLITS * Wp);
  HSG_ALLOC(c->d_beta, sizeof(float) * n_samples * Wp);
  HSG_ALLOC(c->d_temps, sizeof(double) * n_samples * n_temps);
  HSG_ALLOC(c->d_inv_temps, sizeof(double) * n_samples * n_temps);
  HSG_ALLOC(c->d_perm, sizeof(int) * n_samples * n_replicas * n_temps);
  HSG_ALLOC(c->d_E, sizeof(double) * n_samples * Wp);
  HSG_ALLOC(c->d_acc, sizeof(unsigned long long) * n_samples * n_replicas * std::max(1, n_temps - 1));
  HSG_ALLOC(c->d_counters, sizeof(unsigned long long) * 2 * n_samples);
  HSG_ALLOC(c->d_active, sizeof(unsigned char) * n_samples);
  HSG_ALLOC(c->d_bar, sizeof(unsigned int) * 8);
  HSG_ALLOC(c->d_moved, sizeof(unsigned long long) * n_samples * n_replicas * n_temps);
  HSG_ALLOC(c->d_tstate, sizeof(unsigned char) * n_samples * n_replicas * n_temps);
  HSG_ALLOC(c->d_tunnel, sizeof(unsigned int) * n_samples * n_replicas * n_temps);
#undef HSG_ALLOC

  std::vector<double> inv(n_samples * (size_t)n_temps);
  std::vector<float> beta(n_samples * (size_t)Wp, 1.0f);
  std::vector<int> perm(n_samples * (size_t)n_replicas * n_temps);
  for (int s = 0; s < n_samples; ++s) {
    for (int t = 0; t < n_temps; ++t) inv[(size_t)s * n_temps + t] = 1.0 / temps[(size_t)s * n_temps + t];
    for (int r = 0; r < n_replicas; ++r)
      for (int t = 0; t < n_temps; ++t) {
        perm[((size_t)s * n_replicas + r) * n_temps + t] = t;
        beta[(size_t)s * Wp + r * n_temps + t] = (float)inv[(size_t)s * n_temps + t];
      }
  }
  // tunnelling state: the configuration at T_1 (memory slot 0 of each chain) starts at that end
  std::vector<unsigned char> tstate(perm.size(), 0);
  for (size_t k = 0; k < tstate.size(); k += n_temps) tstate[k] = 1;
  c->seed = seed;
  {
    // FNV-1a over what a checkpoint must agree on: sizes, temperatures, records
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](const void* d, size_t n) {
      const unsigned char* b = (const unsigned char*)d;
      for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    };
    mix(L, sizeof(int) * n_samples);
    mix(temps, sizeof(double) * n_samples * n_temps);
    const int dims[4] = {n_temps, n_replicas, opt.precision, opt.j_fp16 ? 1 : 0};
    mix(dims, sizeof(dims));
    if (c->j16) mix(rech.data(), rech.size() * sizeof(__half));
    else mix(recf.data(), recf.size() * sizeof(float));
    c->shape_hash = h;
  }
#define HSG_UP(dst, src, bytes)                                                     \
  e = cudaMemcpy((dst), (src), (bytes), cudaMemcpyHostToDevice);                   \
  if (e != cudaSuccess) {                                                          \
    c->msg = std::string("cudaMemcpy: ") + cudaGetErrorString(e);                  \
    return cleanup_fail(HSG_ECUDA);                                                \
  }
  HSG_UP(c->rec, c->j16 ? (const void*)rech.data() : (const void*)recf.data(), c->rec_bytes);
  HSG_UP(c->d_sd, c->sd.data(), sizeof(SampleDev) * n_samples);
  HSG_UP(c->d_conv_blocks, conv_blocks.data(), sizeof(int4) * conv_blocks.size());
  HSG_UP(c->d_temps, temps, sizeof(double) * n_samples * n_temps);
  HSG_UP(c->d_inv_temps, inv.data(), sizeof(double) * inv.size());
  HSG_UP(c->d_perm, perm.data(), sizeof(int) * perm.size());
  HSG_UP(c->d_beta, beta.data(), sizeof(float) * beta.size());
  {
    const std::vector<unsigned long long> zeros(2 * (size_t)n_samples, 0ull);
    const std::vector<unsigned char> ones((size_t)n_samples, 1);
    HSG_UP(c->d_counters, zeros.data(), sizeof(unsigned long long) * zeros.size());
    HSG_UP(c->d_active, ones.data(), ones.size());
  }
  HSG_UP(c->d_tstate, tstate.data(), tstate.size());
#undef HSG_UP
  e = cudaMemset(c->d_acc, 0, sizeof(unsigned long long) * n_samples * n_replicas * std::max(1, n_temps - 1));
  if (e == cudaSuccess) e = cudaMemset(c->d_moved, 0, sizeof(unsigned long long) * perm.size());
  if (e == cudaSuccess) e = cudaMemset(c->d_tunnel, 0, sizeof(unsigned int) * perm.size());
  if (e == cudaSuccess) e = cudaMemset(c->d_E, 0, sizeof(double) * n_samples * Wp);
  if (e == cudaSuccess) e = cudaMemset(c->d_bar, 0, sizeof(unsigned int) * 8);
  if (e == cudaSuccess) e = cudaMemset(c->spins, 0, c->spin_bytes);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    c->msg = std::string("device init: ") + cudaGetErrorString(e);
    return cleanup_fail(HSG_ECUDA);
  }
  // step schedule: automatic contexts are tuned at their first hsg_step; until
  // then (and for explicit choices) the two-pass graph or the requested one
  {
    c->tune_pending = opt.variant == HSG_VARIANT_AUTO && opt.n_or_per_step >= 1;
    int want = opt.variant == HSG_VARIANT_AUTO ? HSG_VARIANT_TWO_PASS : opt.variant;
    if (opt.n_or_per_step < 1) want = HSG_VARIANT_TWO_PASS;
    c->inject_fault = opt.inject_barrier_fault != 0;
    c->fused_possible = fmt != FMT_YX4;
    for (int s = 0; s < n_samples; ++s)
      if (L[s] % 4 != 0 || L[s] < 8) c->fused_possible = false;
    c->wave_possible = fmt_has_wave(fmt);
    c->staged_possible = c->wave_possible;
    for (int s = 0; s < n_samples; ++s) {
      c->staged_possible = c->staged_possible && lattice_has_staged(L[s]);
      c->Lh_max = std::max(c->Lh_max, L[s] / 2);
    }
    const int sweep = opt.sweep_kernel == HSG_SWEEP_AUTO ? HSG_SWEEP_HALF : opt.sweep_kernel;
    hsg_status st2 = configure_schedule(c, want, c->GPT, opt.pass_bytes, sweep, opt.wave_lag);
    if (st2 != HSG_OK) return cleanup_fail(st2);
  }
  ConvParams cp = conv_params(c, nullptr, nullptr);
  e = launch_init(c->fmt, cp, c->n_conv_blocks, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    c->msg = std::string("init kernel: ") + cudaGetErrorString(e);
    return cleanup_fail(HSG_ECUDA);
  }
  *out = c;
  return HSG_OK;
}

}  // namespace

namespace hsg {
// error text for calls that have no context (reported by hsg_last_error(NULL))
void set_global_error(const char* msg) { g_create_error = msg ? msg : ""; }
}  // namespace hsg

extern "C" {

void hsg_default_options(hsg_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = HSG_FP32;
  opt->n_hb_per_step = 1;
  opt->n_or_per_step = 5;
  opt->barrier_timeout_ms = 2000;
}

hsg_status hsg_create(hsg_ctx** out, int L, const double* temps, int n_temps, int n_replicas,
                      const float* J, const float* H, uint64_t seed, const hsg_options* opt) {
  NvtxRange nvtx_("hsg_create");
  const float* Jp[1] = {J};
  const float* Hp[1] = {H};
  return create_impl(out, 1, &L, temps, n_temps, n_replicas, Jp, Hp, seed, opt);
}

hsg_status hsg_create_batch(hsg_ctx** out, int n_samples, const int* L, const double* temps,
                            int n_temps, int n_replicas, const float* const* J,
                            const float* const* H, uint64_t seed, const hsg_options* opt) {
  NvtxRange nvtx_("hsg_create_batch");
  return create_impl(out, n_samples, L, temps, n_temps, n_replicas, J, H, seed, opt);
}

hsg_status hsg_sweep_or(hsg_ctx* c, int n) {
  NvtxRange nvtx_("hsg_sweep_or");
  HSG_CHECK_CTX(c);
  if (n < 0) return bad_arg(c, "n_sweeps < 0");
  if (n == 0) return HSG_OK;
  HSG_CUDA(c, cudaSetDevice(c->device));
  c->e_valid = false;
  HSG_TRY(or_sweeps(c, n, 0));
  HSG_CUDA(c, launch_bump(c->d_counters, c->d_active, c->ns, n, 0, c->stream));
  return HSG_OK;
}

hsg_status hsg_sweep_hb(hsg_ctx* c, int n) {
  NvtxRange nvtx_("hsg_sweep_hb");
  HSG_CHECK_CTX(c);
  if (n < 0) return bad_arg(c, "n_sweeps < 0");
  if (n == 0) return HSG_OK;
  HSG_CUDA(c, cudaSetDevice(c->device));
  c->e_valid = false;
  for (int k = 0; k < n; ++k) HSG_TRY(half_sweeps(c, true, k));
  HSG_CUDA(c, launch_bump(c->d_counters, c->d_active, c->ns, n, 0, c->stream));
  return HSG_OK;
}

hsg_status hsg_pt_exchange(hsg_ctx* c) {
  NvtxRange nvtx_("hsg_pt_exchange");
  HSG_CHECK_CTX(c);
  HSG_CUDA(c, cudaSetDevice(c->device));
  HSG_TRY(enqueue_energy(c));
  c->e_valid = true;
  HSG_CUDA(c, launch_pt(pt_params(c, 0, 1), c->stream));
  return HSG_OK;
}

hsg_status hsg_pt_exchange_energies(hsg_ctx* c, const double* E_sys) {
  NvtxRange nvtx_("hsg_pt_exchange_energies");
  HSG_CHECK_CTX(c);
  if (!E_sys) return bad_arg(c, "E_sys is NULL");
  HSG_CUDA(c, cudaSetDevice(c->device));
  HSG_CUDA(c, cudaMemcpy2DAsync(c->d_E, sizeof(double) * c->Wp, E_sys, sizeof(double) * c->W,
                                sizeof(double) * c->W, c->ns, cudaMemcpyHostToDevice, c->stream));
  c->e_valid = false;   // the caller's energies need not be those of the state
  HSG_CUDA(c, launch_pt(pt_params(c, 0, 1), c->stream));
  // the host array may be released by the caller on return
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  return HSG_OK;
}

// The block table of the multi-hit schedule for tile edge T (index 0: T = 4,
// 1: T = 8): every (tile, chunk group) of colour 0 of every sample, then those
// of colour 1.
static hsg_status multihit_table(hsg_ctx* c, int T) {
  const int ti = T == 4 ? 0 : 1;
  if (c->d_mh_blocks[ti]) return HSG_OK;
  std::vector<int4> blocks;
  for (int color = 0; color < 2; ++color) {
    const size_t before = blocks.size();
    for (int s = 0; s < c->ns; ++s) {
      const int B = c->L[s] / T;
      for (int t = 0; t < B * B * B; ++t) {
        if (((t % B + (t / B) % B + t / (B * B)) & 1) != color) continue;
        for (int g = 0; g < c->G; ++g) blocks.push_back(make_int4(s, t, g, 0));
      }
    }
    c->mh_count[ti][color] = (int)(blocks.size() - before);
  }
  HSG_TRY(dev_alloc(c, &c->d_mh_blocks[ti], sizeof(int4) * blocks.size()));
  HSG_CUDA(c, cudaMemcpy(c->d_mh_blocks[ti], blocks.data(), sizeof(int4) * blocks.size(),
                         cudaMemcpyHostToDevice));
  return HSG_OK;
}

hsg_status hsg_step_multihit(hsg_ctx* c, int n_steps, int tile, int n_rounds, int n_or, int n_hb) {
  NvtxRange nvtx_("hsg_step_multihit");
  HSG_CHECK_CTX(c);
  if (n_steps < 0) return bad_arg(c, "n_steps < 0");
  if (tile != 4 && tile != 8) return bad_arg(c, "tile must be 4 or 8");
  if (n_rounds < 1 || n_or < 0 || n_hb < 0 || n_or + n_hb < 1)
    return bad_arg(c, "need n_rounds >= 1, n_or >= 0, n_hb >= 0 and n_or + n_hb >= 1");
  for (int s = 0; s < c->ns; ++s)
    if (c->L[s] % (2 * tile) != 0) return bad_arg(c, "every L must be a multiple of 2 * tile");
  if (n_steps == 0) return HSG_OK;
  HSG_CUDA(c, cudaSetDevice(c->device));
  HSG_TRY(multihit_table(c, tile));
  const int ti = tile == 4 ? 0 : 1;
  MultihitParams p;
  p.spins = c->spins;
  p.rec = c->rec;
  p.samples = c->d_sd;
  p.blocks = c->d_mh_blocks[ti];
  p.beta = c->d_beta;
  p.counters = c->d_counters;
  p.active = c->d_active;
  p.Wp = c->Wp;
  p.n_rounds = n_rounds;
  p.n_or = n_or;
  p.n_hb = n_hb;
  const SweepParams sp = sweep_params(c, 0, 0);
  for (int r = 0; r < 20; ++r) p.rk[r] = sp.rk[r];
  const bool fast = c->opt.fast_math != 0;
  for (int k = 0; k < n_steps; ++k) {
    for (int color = 0; color < 2; ++color) {
      p.blk_base = color == 0 ? 0 : c->mh_count[ti][0];
      HSG_CUDA(c, launch_multihit(c->fmt, c->j16, fast, tile, p, c->mh_count[ti][color], c->stream));
    }
    HSG_TRY(enqueue_energy(c));
    HSG_CUDA(c, launch_pt(pt_params(c, n_rounds * (n_or + n_hb), 1), c->stream));
  }
  c->e_valid = true;
  return HSG_OK;
}

hsg_status hsg_step(hsg_ctx* c, int n_steps) {
  NvtxRange nvtx_("hsg_step");
  HSG_CHECK_CTX(c);
  if (n_steps < 0) return bad_arg(c, "n_steps < 0");
  if (n_steps == 0) return HSG_OK;
  HSG_CUDA(c, cudaSetDevice(c->device));
  if (c->tune_pending) HSG_TRY(autotune(c));
  HSG_TRY(run_steps(c, n_steps));
  c->e_valid = true;    // every step ends with the energies of its final state
  return HSG_OK;
}

hsg_status hsg_energies(hsg_ctx* c, double* E_sys) {
  NvtxRange nvtx_("hsg_energies");
  HSG_CHECK_CTX(c);
  if (!E_sys) return bad_arg(c, "E_sys is NULL");
  HSG_CUDA(c, cudaSetDevice(c->device));
  HSG_TRY(enqueue_energy(c));
  c->e_valid = true;
  HSG_CUDA(c, cudaMemcpy2DAsync(E_sys, sizeof(double) * c->W, c->d_E, sizeof(double) * c->Wp,
                                sizeof(double) * c->W, c->ns, cudaMemcpyDeviceToHost, c->stream));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  return HSG_OK;
}

hsg_status hsg_last_energies(hsg_ctx* c, double* E_sys) {
  HSG_CHECK_CTX(c);
  if (!E_sys) return bad_arg(c, "E_sys is NULL");
  HSG_CUDA(c, cudaSetDevice(c->device));
  HSG_CUDA(c, cudaMemcpy2DAsync(E_sys, sizeof(double) * c->W, c->d_E, sizeof(double) * c->Wp,
                                sizeof(double) * c->W, c->ns, cudaMemcpyDeviceToHost, c->stream));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  return HSG_OK;
}

// Parameters common to the measurement launches; g.ok selects the staged
// kernels (geometry from staged_geometry), otherwise the direct ones.
static OverlapParams overlap_params(hsg_ctx* c, const StagedGeom& g) {
  OverlapParams p{};
  p.spins = c->spins;
  p.samples = c->d_sd;
  p.perm = c->d_perm;
  p.n_samples = c->ns;
  p.R_O = c->R_O;
  p.R_T = c->R_T;
  p.Wp = c->Wp;
  if (g.ok) {
    p.sub = g.sub;
    p.tile_ss = g.tile_ss;
    p.Gu = g.Gu;
    p.grow = g.grow;
  }
  p.err = c->d_bar + 3;
  p.timeout_ns = (unsigned long long)std::max(1, c->opt.barrier_timeout_ms) * 1000000ull;
  return p;
}

hsg_status hsg_measure(hsg_ctx* c, hsg_obs* o) {
  NvtxRange nvtx_("hsg_measure");
  HSG_CHECK_CTX(c);
  if (!o) return bad_arg(c, "obs is NULL");
  HSG_CUDA(c, cudaSetDevice(c->device));
  // the energies a step leaves behind are those of its final state
  if (!c->e_valid) HSG_TRY(enqueue_energy(c));
  c->e_valid = true;
  const bool pairs = c->R_O >= 2 && (o->q || o->qk);
  if (pairs) {
    const long long nmax = (long long)c->Lmax * c->Lmax * c->Lmax;
    const StagedGeom g = staged_geometry(c->fmt, true, c->R_O, c->R_T, nmax, c->total_sites);
    const int n_tiles = g.ok ? g.n_tiles : (int)((nmax + MEAS_TILE - 1) / MEAS_TILE);
    if (!c->d_mpart) {
      const size_t vals = g.ok ? (size_t)n_tiles * g.values
                               : (size_t)3 * n_tiles * meas_partial_values(true, false);
      HSG_TRY(dev_alloc(c, &c->d_mpart, sizeof(double) * c->ns * (size_t)c->R_T * vals));
      HSG_TRY(dev_alloc(c, &c->d_q, sizeof(double) * c->ns * (size_t)c->R_T * 9));
      HSG_TRY(dev_alloc(c, &c->d_qk, sizeof(double) * c->ns * (size_t)c->R_T * 54));
    }
    OverlapParams p = overlap_params(c, g);
    p.partials = c->d_mpart;
    p.D = c->d_q;
    p.C = c->d_qk;
    p.n_pairs = 3;          // direct kernel: units are the rows mu of the tensor
    p.n_tiles = n_tiles;
    HSG_CUDA(c, launch_qtensor(c->fmt, p, c->stream));
  }
  std::vector<double> E((size_t)c->ns * c->Wp);
  std::vector<int> perm((size_t)c->ns * c->R_O * c->R_T);
  HSG_CUDA(c, cudaMemcpyAsync(E.data(), c->d_E, sizeof(double) * E.size(), cudaMemcpyDeviceToHost,
                              c->stream));
  HSG_CUDA(c, cudaMemcpyAsync(perm.data(), c->d_perm, sizeof(int) * perm.size(),
                              cudaMemcpyDeviceToHost, c->stream));
  if (pairs && o->q)
    HSG_CUDA(c, cudaMemcpyAsync(o->q, c->d_q, sizeof(double) * c->ns * c->R_T * 9,
                                cudaMemcpyDeviceToHost, c->stream));
  if (pairs && o->qk)
    HSG_CUDA(c, cudaMemcpyAsync(o->qk, c->d_qk, sizeof(double) * c->ns * c->R_T * 54,
                                cudaMemcpyDeviceToHost, c->stream));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  for (int s = 0; s < c->ns; ++s)
    for (int r = 0; r < c->R_O; ++r)
      for (int t = 0; t < c->R_T; ++t) {
        const size_t pi = ((size_t)s * c->R_O + r) * c->R_T + t;
        if (o->E) o->E[pi] = E[(size_t)s * c->Wp + r * c->R_T + perm[pi]];
        if (o->perm) o->perm[pi] = perm[pi];
      }
  return HSG_OK;
}

hsg_status hsg_get_spins_dev(hsg_ctx* c, float* xyz_dev) {
  HSG_CHECK_CTX(c);
  if (!xyz_dev) return bad_arg(c, "xyz is NULL");
  HSG_CUDA(c, cudaSetDevice(c->device));
  HSG_TRY(ensure_xyz(c));
  HSG_CUDA(c, launch_get(c->fmt, conv_params(c, xyz_dev, c->d_xyz_off), c->n_conv_blocks, c->stream));
  return HSG_OK;
}

hsg_status hsg_set_spins_dev(hsg_ctx* c, const float* xyz_dev) {
  HSG_CHECK_CTX(c);
  if (!xyz_dev) return bad_arg(c, "xyz is NULL");
  HSG_CUDA(c, cudaSetDevice(c->device));
  HSG_TRY(ensure_xyz(c));
  HSG_CUDA(c, launch_set(c->fmt, conv_params(c, const_cast<float*>(xyz_dev), c->d_xyz_off),
                         c->n_conv_blocks, c->stream));
  c->e_valid = false;
  return HSG_OK;
}

// Replica pairs of the overlap measurements: all pairs of the first
// min(n_replicas, 4) replicas.
int overlap_pairs(int R_O) {
  const int r = std::min(R_O, 4);
  return r * (r - 1) / 2;
}

// The chirality buffer of the staged chiral overlaps: per sample three planes
// (a = x, y, z) of Gu chunk groups x N sites x 16 bytes.
static hsg_status ensure_kappa(hsg_ctx* c, int Gu) {
  if (c->d_kappa) return HSG_OK;
  std::vector<SampleDev> kd(c->sd);
  size_t off = 0;
  for (int s = 0; s < c->ns; ++s) {
    kd[s].plane_stride = (long long)Gu * c->sd[s].N * 16;
    kd[s].spin_off = (long long)off;
    off += (size_t)(3 * kd[s].plane_stride + 255) / 256 * 256;
  }
  HSG_TRY(dev_alloc(c, &c->d_kappa, off));
  HSG_TRY(dev_alloc(c, &c->d_sd_k, sizeof(SampleDev) * c->ns));
  HSG_CUDA(c, cudaMemcpy(c->d_sd_k, kd.data(), sizeof(SampleDev) * c->ns, cudaMemcpyHostToDevice));
  return HSG_OK;
}

hsg_status hsg_measure_overlaps(hsg_ctx* c, double* D, double* C) {
  NvtxRange nvtx_("hsg_measure_overlaps");
  HSG_CHECK_CTX(c);
  if (!D && !C) return bad_arg(c, "D and C are both NULL");
  if (c->R_O < 2) return bad_arg(c, "overlaps need n_replicas >= 2");
  HSG_CUDA(c, cudaSetDevice(c->device));
  const int n_pairs = overlap_pairs(c->R_O);
  const long long nmax = (long long)c->Lmax * c->Lmax * c->Lmax;
  const int n_tiles = (int)((nmax + MEAS_TILE - 1) / MEAS_TILE);
  // D: the staged kernel over the spins.  C: the chiralities of every site
  // into a binary32 buffer, then the staged kernel over that buffer.  Either
  // falls back to the direct kernel when its staged systems exceed shared memory.
  const StagedGeom g = staged_geometry(c->fmt, false, c->R_O, c->R_T, nmax, c->total_sites);
  const StagedGeom gk = staged_geometry(FMT_F32, false, c->R_O, c->R_T, nmax, c->total_sites);
  if (!c->d_opart) {
    const size_t direct = (size_t)n_pairs * n_tiles * meas_partial_values(false, true);
    const size_t staged = g.ok ? (size_t)g.n_tiles * g.values : 0;
    const size_t staged_c = gk.ok ? (size_t)gk.n_tiles * 3 * gk.values : 0;
    HSG_TRY(dev_alloc(c, &c->d_opart, sizeof(double) * c->ns * (size_t)c->R_T *
                                          std::max(direct, std::max(staged, staged_c))));
    HSG_TRY(dev_alloc(c, &c->d_D, sizeof(double) * c->ns * (size_t)c->R_T * n_pairs * 8));
    HSG_TRY(dev_alloc(c, &c->d_C, sizeof(double) * c->ns * (size_t)c->R_T * n_pairs * 24));
  }
  if (C && gk.ok) {
    HSG_TRY(ensure_kappa(c, gk.Gu));
    for (int parity = 0; parity < 2; ++parity) {
      ChiralityParams kp;
      kp.spins = c->spins;
      kp.kappa = c->d_kappa;
      kp.samples = c->d_sd;
      kp.ksamples = c->d_sd_k;
      kp.blocks = c->d_sweep_blocks;
      kp.G = c->G;
      kp.GPT = c->GPT;
      kp.Gu = gk.Gu;
      kp.parity = parity;
      HSG_CUDA(c, launch_chirality(c->fmt, kp, c->n_sweep_blocks, c->stream));
    }
    OverlapParams pc = overlap_params(c, gk);
    pc.spins = c->d_kappa;
    pc.samples = c->d_sd_k;
    pc.partials = c->d_opart;
    pc.C = c->d_C;
    pc.n_pairs = n_pairs;
    pc.n_tiles = gk.n_tiles;
    HSG_CUDA(c, launch_chiral_staged(pc, c->stream));
  }
  const bool direct_c = C && !gk.ok;       // the direct kernel gives D and C together
  if (D || direct_c) {
    const bool staged = g.ok && !direct_c;
    OverlapParams p = overlap_params(c, staged ? g : StagedGeom{});
    p.partials = c->d_opart;
    p.D = c->d_D;
    p.C = direct_c ? c->d_C : nullptr;
    p.n_pairs = n_pairs;
    p.n_tiles = staged ? g.n_tiles : n_tiles;
    HSG_CUDA(c, launch_overlaps(c->fmt, p, direct_c, c->stream));
  }
  if (D)
    HSG_CUDA(c, cudaMemcpyAsync(D, c->d_D, sizeof(double) * c->ns * c->R_T * n_pairs * 8,
                                cudaMemcpyDeviceToHost, c->stream));
  if (C)
    HSG_CUDA(c, cudaMemcpyAsync(C, c->d_C, sizeof(double) * c->ns * c->R_T * n_pairs * 24,
                                cudaMemcpyDeviceToHost, c->stream));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  return HSG_OK;
}

hsg_status hsg_get_spins(hsg_ctx* c, float* xyz) {
  NvtxRange nvtx_("hsg_get_spins");
  HSG_CHECK_CTX(c);
  if (!xyz) return bad_arg(c, "xyz is NULL");
  HSG_CUDA(c, cudaSetDevice(c->device));
  HSG_TRY(ensure_xyz(c));
  HSG_CUDA(c, launch_get(c->fmt, conv_params(c, c->d_xyz, c->d_xyz_off), c->n_conv_blocks, c->stream));
  HSG_CUDA(c, cudaMemcpyAsync(xyz, c->d_xyz, sizeof(float) * c->xyz_floats, cudaMemcpyDeviceToHost,
                              c->stream));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  return HSG_OK;
}

hsg_status hsg_set_spins(hsg_ctx* c, const float* xyz) {
  NvtxRange nvtx_("hsg_set_spins");
  HSG_CHECK_CTX(c);
  if (!xyz) return bad_arg(c, "xyz is NULL");
  HSG_CUDA(c, cudaSetDevice(c->device));
  HSG_TRY(ensure_xyz(c));
  HSG_CUDA(c, cudaMemcpyAsync(c->d_xyz, xyz, sizeof(float) * c->xyz_floats, cudaMemcpyHostToDevice,
                              c->stream));
  HSG_CUDA(c, launch_set(c->fmt, conv_params(c, c->d_xyz, c->d_xyz_off), c->n_conv_blocks, c->stream));
  c->e_valid = false;
  // the host buffer has been read once the copy is done
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  return HSG_OK;
}

hsg_status hsg_get_perm(hsg_ctx* c, int32_t* perm) {
  HSG_CHECK_CTX(c);
  if (!perm) return bad_arg(c, "perm is NULL");
  HSG_CUDA(c, cudaSetDevice(c->device));
  HSG_CUDA(c, cudaMemcpyAsync(perm, c->d_perm, sizeof(int) * c->ns * c->R_O * c->R_T,
                              cudaMemcpyDeviceToHost, c->stream));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  return HSG_OK;
}

hsg_status hsg_get_pt_stats(hsg_ctx* c, uint64_t* accepted, uint64_t* n_calls) {
  HSG_CHECK_CTX(c);
  HSG_CUDA(c, cudaSetDevice(c->device));
  unsigned long long cnt[2];
  if (accepted && c->R_T > 1)
    HSG_CUDA(c, cudaMemcpyAsync(accepted, c->d_acc,
                                sizeof(unsigned long long) * c->ns * c->R_O * (c->R_T - 1),
                                cudaMemcpyDeviceToHost, c->stream));
  HSG_CUDA(c, cudaMemcpyAsync(cnt, c->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  if (n_calls) *n_calls = cnt[1];
  return HSG_OK;
}

hsg_status hsg_set_active(hsg_ctx* c, const uint8_t* active) {
  HSG_CHECK_CTX(c);
  HSG_CUDA(c, cudaSetDevice(c->device));
  std::vector<unsigned char> a((size_t)c->ns, 1);
  if (active)
    for (int s = 0; s < c->ns; ++s) a[s] = active[s] ? 1 : 0;
  HSG_CUDA(c, cudaMemcpyAsync(c->d_active, a.data(), a.size(), cudaMemcpyHostToDevice, c->stream));
  // the host array may be released on return
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  return HSG_OK;
}

hsg_status hsg_get_counters(hsg_ctx* c, uint64_t* sweeps, uint64_t* pt_passes) {
  HSG_CHECK_CTX(c);
  HSG_CUDA(c, cudaSetDevice(c->device));
  std::vector<unsigned long long> cnt(2 * (size_t)c->ns);
  HSG_CUDA(c, cudaMemcpyAsync(cnt.data(), c->d_counters, sizeof(unsigned long long) * cnt.size(),
                              cudaMemcpyDeviceToHost, c->stream));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  for (int s = 0; s < c->ns; ++s) {
    if (sweeps) sweeps[s] = cnt[2 * (size_t)s];
    if (pt_passes) pt_passes[s] = cnt[2 * (size_t)s + 1];
  }
  return HSG_OK;
}

hsg_status hsg_get_pt_diagnostics(hsg_ctx* c, uint64_t* moved, uint32_t* tunnel, uint64_t* n_passes) {
  HSG_CHECK_CTX(c);
  HSG_CUDA(c, cudaSetDevice(c->device));
  const size_t n = (size_t)c->ns * c->R_O * c->R_T;
  unsigned long long cnt[2];
  if (moved)
    HSG_CUDA(c, cudaMemcpyAsync(moved, c->d_moved, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, c->stream));
  if (tunnel)
    HSG_CUDA(c, cudaMemcpyAsync(tunnel, c->d_tunnel, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, c->stream));
  HSG_CUDA(c, cudaMemcpyAsync(cnt, c->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  if (n_passes) *n_passes = cnt[1];
  return HSG_OK;
}

namespace {
// checkpoint blob: this header, the stored spins as they are in device memory,
// then the chain-state regions in chain_regions order
struct CheckpointHeader {
  char magic[8];
  uint32_t version;
  uint32_t fmt, j16, ns, R_O, R_T, W, Wp, e_valid;
  uint64_t seed, shape_hash, spin_bytes, state_bytes;
};
const char kMagic[8] = {'H', 'S', 'G', 'C', 'K', 'P', 'T', '1'};
}  // namespace

hsg_status hsg_checkpoint_size(hsg_ctx* c, size_t* bytes) {
  HSG_CHECK_CTX(c);
  if (!bytes) return bad_arg(c, "bytes is NULL");
  *bytes = sizeof(CheckpointHeader) + c->spin_bytes + chain_state_bytes(c);
  return HSG_OK;
}

hsg_status hsg_checkpoint_save(hsg_ctx* c, void* buf, size_t bytes) {
  NvtxRange nvtx_("hsg_checkpoint_save");
  HSG_CHECK_CTX(c);
  if (!buf) return bad_arg(c, "buf is NULL");
  const size_t need = sizeof(CheckpointHeader) + c->spin_bytes + chain_state_bytes(c);
  if (bytes < need) return bad_arg(c, "checkpoint buffer too small");
  HSG_CUDA(c, cudaSetDevice(c->device));
  CheckpointHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, 8);
  h.version = 1;
  h.fmt = (uint32_t)c->fmt;
  h.j16 = c->j16 ? 1u : 0u;
  h.ns = (uint32_t)c->ns;
  h.R_O = (uint32_t)c->R_O;
  h.R_T = (uint32_t)c->R_T;
  h.W = (uint32_t)c->W;
  h.Wp = (uint32_t)c->Wp;
  h.e_valid = c->e_valid ? 1u : 0u;
  h.seed = c->seed;
  h.shape_hash = c->shape_hash;
  h.spin_bytes = c->spin_bytes;
  h.state_bytes = chain_state_bytes(c);
  unsigned char* out = (unsigned char*)buf;
  std::memcpy(out, &h, sizeof(h));
  HSG_CUDA(c, cudaMemcpyAsync(out + sizeof(h), c->spins, c->spin_bytes, cudaMemcpyDeviceToHost, c->stream));
  HSG_TRY(copy_chain_state(c, out + sizeof(h) + c->spin_bytes, true));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  return HSG_OK;
}

hsg_status hsg_checkpoint_load(hsg_ctx* c, const void* buf, size_t bytes) {
  NvtxRange nvtx_("hsg_checkpoint_load");
  HSG_CHECK_CTX(c);
  if (!buf) return bad_arg(c, "buf is NULL");
  if (bytes < sizeof(CheckpointHeader)) return bad_arg(c, "checkpoint too short");
  CheckpointHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != 1) return bad_arg(c, "not a checkpoint");
  if (h.fmt != (uint32_t)c->fmt || h.j16 != (c->j16 ? 1u : 0u) || h.ns != (uint32_t)c->ns ||
      h.R_O != (uint32_t)c->R_O || h.R_T != (uint32_t)c->R_T || h.W != (uint32_t)c->W ||
      h.Wp != (uint32_t)c->Wp || h.seed != c->seed || h.shape_hash != c->shape_hash ||
      h.spin_bytes != c->spin_bytes || h.state_bytes != chain_state_bytes(c))
    return bad_arg(c, "checkpoint of a different context shape, disorder, precision or seed");
  if (bytes < sizeof(h) + h.spin_bytes + h.state_bytes) return bad_arg(c, "checkpoint truncated");
  HSG_CUDA(c, cudaSetDevice(c->device));
  const unsigned char* in = (const unsigned char*)buf;
  HSG_CUDA(c, cudaMemcpyAsync(c->spins, in + sizeof(h), c->spin_bytes, cudaMemcpyHostToDevice, c->stream));
  HSG_TRY(copy_chain_state(c, const_cast<unsigned char*>(in) + sizeof(h) + c->spin_bytes, false));
  // the host buffer may be released on return
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  c->e_valid = h.e_valid != 0;
  return HSG_OK;
}

hsg_status hsg_get_info(hsg_ctx* c, hsg_info* info) {
  HSG_CHECK_CTX(c);
  if (!info) return bad_arg(c, "info is NULL");
  HSG_CUDA(c, cudaSetDevice(c->device));
  unsigned long long cnt[2];
  HSG_CUDA(c, cudaMemcpyAsync(cnt, c->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  info->n_samples = c->ns;
  info->n_temps = c->R_T;
  info->n_replicas = c->R_O;
  info->W = c->W;
  info->Wp = c->Wp;
  info->precision = c->fmt;
  info->j_fp16 = c->j16 ? 1 : 0;
  info->variant = c->variant;
  info->chunks_per_thread = c->GPT;
  info->n_passes = (int)c->pass_bound.size() - 1;
  info->n_overlap_pairs = c->R_O >= 2 ? overlap_pairs(c->R_O) : 0;
  info->pass_bytes = c->pass_bytes;
  info->total_sites = c->total_sites;
  info->total_spins = c->total_sites * c->W;
  info->spin_bytes = (long long)c->spin_bytes;
  info->rec_bytes = (long long)c->rec_bytes;
  info->sweep_count = cnt[0];
  info->pt_count = cnt[1];
  info->stream = (void*)c->stream;
  info->sweep_kernel = c->use_wave ? HSG_SWEEP_WAVE
                      : c->use_staged ? HSG_SWEEP_STAGED
                      : (c->use_fused ? HSG_SWEEP_FUSED : HSG_SWEEP_HALF);
  info->staged = (c->use_wave && c->staged_possible) || c->use_staged;
  info->wave_lag = c->use_wave ? c->wave_lag : 0;
  info->fused_band_rows = c->fused_ny.empty() ? 0 : c->fused_ny[0];
  info->fused_items = c->n_fused_items;
  return HSG_OK;
}

hsg_status hsg_sync(hsg_ctx* c) {
  HSG_CHECK_CTX(c);
  HSG_CUDA(c, cudaSetDevice(c->device));
  HSG_CUDA(c, cudaStreamSynchronize(c->stream));
  HSG_TRY(poll_device_error(c));
  HSG_CUDA(c, cudaGetLastError());
  return HSG_OK;
}

hsg_status hsg_philox(const uint32_t* ctr, long long n, uint64_t seed, uint32_t* out) {
  if (!ctr || !out || n < 0) {
    g_create_error = "bad arguments to hsg_philox";
    return HSG_EINVAL;
  }
  if (n == 0) return HSG_OK;
  SweepParams p{};
  uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    p.rk[2 * r] = k0;
    p.rk[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  uint4 *dc = nullptr, *dout = nullptr;
  const size_t bytes = sizeof(uint4) * (size_t)n;
  cudaError_t e = cudaMalloc(&dc, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&dout, bytes);
  if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_philox(dc, n, p, dout, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost);
  if (dc) cudaFree(dc);
  if (dout) cudaFree(dout);
  if (e != cudaSuccess) {
    g_create_error = std::string("hsg_philox: ") + cudaGetErrorString(e);
    return HSG_ECUDA;
  }
  return HSG_OK;
}

const char* hsg_last_error(const hsg_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->msg.c_str();
}

const char* hsg_status_string(hsg_status st) {
  switch (st) {
    case HSG_OK: return "ok";
    case HSG_EINVAL: return "invalid argument";
    case HSG_ENOMEM: return "out of memory";
    case HSG_ECUDA: return "CUDA error";
    case HSG_ETIMEOUT: return "device wait timed out";
    case HSG_ESTATE: return "invalid state";
  }
  return "unknown status";
}

void hsg_destroy(hsg_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  for (void* p : c->allocations) cudaFree(p);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // extern "C"
