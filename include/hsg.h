/*
 * hsg — Heisenberg spin-glass Monte Carlo on one GB300 (sm_103a).
 *
 * C ABI of the CUDA library libhsg.so.  It runs the hot path of the method of
 * Yavors'kii & Weigel, "Optimized GPU simulation of continuous-spin glass
 * models" (arXiv:1204.6192): checkerboard heat-bath (HB) and over-relaxation
 * (OR) sweeps of the 3D Edwards-Anderson Heisenberg model in a random field,
 * Eq. (1), for many temperatures, replicas and disorder samples at once, the
 * parallel-tempering (PT) exchange of Eq. (4) and the measurements of Eq. (5)
 * and its k-dependent form.  No argument is a framework type: plain pointers
 * and sizes only.
 *
 * Conventions
 *   lattice    L^3 periodic simple cubic, L even and >= 4.  Site index
 *              i = x + L*(y + L*z), parity p(i) = (x + y + z) mod 2.
 *   J          float[N][3], J[i][a] = coupling of the bond (i, i + e_a),
 *              a = x, y, z.  Every bond appears once (Eq. 1 reading).
 *   H          float[N][3] random field, or NULL for H = 0.
 *   systems    a sample (one disorder realisation) holds W = n_replicas *
 *              n_temps systems; system w = r * n_temps + j (replica r, memory
 *              slot j).  All samples of a context have the same n_temps and
 *              n_replicas; their L may differ.  Global system id of sample s:
 *              s * Wp + w with Wp = W rounded up to a multiple of 8.  Global
 *              chain id: s * n_replicas + r.
 *   perm       int32[n_samples][n_replicas][n_temps]: perm[s][r][t] = memory
 *              slot j of replica r that currently holds temperature t.
 *              Initially perm[s][r][t] = t.  PT permutes temperatures, never
 *              spins (Sec. 3.2).
 *   spins      host or device float[...][W][N][3] in sample order: for each
 *              sample, its W systems in memory-slot order, each N sites, each
 *              (x, y, z) components.
 *   random     Philox4x32-10 (Salmon et al., SC'11), key = (seed & 0xffffffff,
 *              seed >> 32); uniforms u(x) = (2*(x >> 9) + 1) * 2^-24.
 *              Initial spins:  counter (i, gsys >> 1, 0, 0)
 *              HB sweep n:     counter (i, gsys >> 1, n, 1)
 *              PT call m:      counter (k, gchain, m, 2), word 0
 *              A system uses words 2*(gsys & 1) and 2*(gsys & 1) + 1.  The
 *              sweep counter n counts every sweep, OR or HB, since creation.
 *   moves      sweep = even half-sweep then odd half-sweep (Sec. 3.1).
 *              OR: s' = 2 (s.h)/(h.h) h - s, s' = s if h = 0 (Eq. 3).
 *              HB: a = beta |h|, d = -log1p((1-u1) expm1(-2a)) / a (a > 1e-12,
 *              else d = 2 (1 - u1)), cos t = 1 - d, sin t = sqrt(d (2 - d)),
 *              azimuth 2 pi u2 in the Duff et al. (JCGT 2017) frame around h
 *              (Eq. 2).  Every move ends with s <- s / |s| and the storage codec.
 *   step       hsg_step: n_hb HB sweeps, n_or OR sweeps, FP64 energies, one PT
 *              pass (Sec. 3.2, steps 1-10 with n_T = 1).
 *
 * Errors: every call returns hsg_status.  The first device error is sticky:
 * later calls on the same context return it until hsg_destroy.  Calls are
 * asynchronous on the context's stream except those that return host data
 * (hsg_get_*, hsg_energies, hsg_measure, hsg_sync), which synchronise.
 * A context must be used from one host thread at a time.
 */
#ifndef HSG_H
#define HSG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hsg_ctx hsg_ctx;   /* opaque, owned by the library */

typedef enum {
  HSG_OK = 0,
  HSG_EINVAL = 1,     /* bad argument (checked on the host before any device work) */
  HSG_ENOMEM = 2,     /* device or host allocation failed */
  HSG_ECUDA = 3,      /* a CUDA call or kernel failed; sticky */
  HSG_ETIMEOUT = 4,   /* a bounded device wait ran out; sticky */
  HSG_ESTATE = 5      /* call not valid in the context's current state */
} hsg_status;

typedef enum {
  HSG_FP32 = 0,       /* 3 x binary32 per spin (12 bytes) */
  HSG_FP16 = 1,       /* 3 x binary16, round to nearest even (6 bytes) */
  HSG_BF16 = 2,       /* 3 x bfloat16, round to nearest even (6 bytes) */
  HSG_ANGLE16 = 3,    /* polar angle and azimuth, 16 bits each (4 bytes) */
  HSG_OCT16 = 4,      /* octahedral map (Cigolle et al. 2014), 16 bits each (4 bytes) */
  HSG_YX4 = 5         /* the paper's packing (Sec. 3.3): binary32 s_y and binary32
                         s_x + 4 sign(s_z) (8 bytes); s_z = sign sqrt(1 - s_x^2 - s_y^2) */
} hsg_precision;

typedef struct {
  int precision;      /* hsg_precision of the stored spins; arithmetic is always FP32 */
  int j_fp16;         /* nonzero: J and H stored as binary16 (rounded to nearest even) */
  int fast_math;      /* nonzero: HB uses the hardware approximate log/exp (Table 1 "fast_math") */
  int n_hb_per_step;  /* HB sweeps per hsg_step (default 1) */
  int n_or_per_step;  /* OR sweeps per hsg_step (default 5) */
  int device;         /* CUDA device ordinal (default 0) */
  void* stream;       /* cudaStream_t to use; NULL: the library creates a non-blocking stream */
  int variant;        /* step schedule: 0 = automatic, else an HSG_VARIANT_* value */
  int barrier_timeout_ms;   /* bound of every device wait: the grid barriers of the
                               persistent schedule, the waits of the measurement kernels
                               for their staged spin copies, of the fused and staged sweeps
                               for their row copies and of the wave sweep for its even blocks
                               (default 2000); a wait that runs
                               out ends the launch and the next synchronising call returns
                               HSG_ETIMEOUT */
  int inject_barrier_fault; /* testing only: nonzero makes one block skip the first grid
                               barrier of the next persistent launch, so the others time out,
                               or (wave sweep, outside hsg_step) makes one odd block of the next
                               hsg_sweep_or launch wait for a flag that no block sets */
  long long pass_bytes;     /* system blocking of hsg_step: the systems are cut into passes
                               (ranges of 4-system chunks, samples kept whole where they fit)
                               of at most this many bytes of spins plus couplings, and each
                               pass runs all sweeps of the step before the next one, so that
                               its later sweeps read the L2 cache.  0 (default): chosen by
                               the automatic schedule, one pass for an explicit variant.
                               Results do not depend on it. */
  int chunks_per_thread;    /* sweep kernels: chunks of 4 systems one thread walks; 0
                               (default): chosen from the problem size (and by the
                               automatic schedule).  Results do not depend on it. */
  int sweep_kernel;         /* over-relaxation sweeps of hsg_step and hsg_sweep_or: an
                               HSG_SWEEP_* value.  HSG_SWEEP_FUSED does both half-sweeps of
                               a sweep in one launch (a wavefront along z through shared
                               memory), pairs of sweeps at a time, reading the spins once
                               and writing them once per sweep; it needs a second spin
                               buffer of spin_bytes, every L a multiple of 4 and a storage
                               format other than HSG_YX4, and is used with the two-pass
                               schedule in one pass (elsewhere the per-half-sweep kernel
                               runs).  HSG_SWEEP_WAVE also does both half-sweeps of a
                               sweep in one launch: the blocks of the per-half-sweep kernel,
                               the odd-parity blocks of each plane following the even-parity
                               blocks of the planes around it, so that they read the spins
                               from the L2 cache; it needs a storage format among HSG_FP32,
                               HSG_FP16 and HSG_BF16 and the two-pass schedule (any pass
                               footprint); where every L is a power of 2 and at least 32,
                               its blocks stage their neighbour rows through shared
                               memory with bulk copies.  HSG_SWEEP_STAGED keeps one launch
                               per half-sweep but with that staged block body (same
                               conditions).  0 (default): chosen by the automatic
                               schedule among the half-sweep, fused and staged kernels
                               (the wave sweep only when requested).  Results do not
                               depend on it (bit for bit). */
  int wave_lag;             /* HSG_SWEEP_WAVE: even-parity blocks scheduled between the last
                               even block an odd block reads and that odd block (more: fewer
                               waits, more spins held in L2).  0 (default): chosen from the
                               number of resident blocks and by the automatic schedule. */
  int inject_alloc_fault;   /* testing only: n > 0 makes the n-th device allocation of the
                               context fail as an out-of-memory would (HSG_ENOMEM; during
                               hsg_create the partial context is released); 0: off */
} hsg_options;

enum {
  HSG_SWEEP_AUTO = 0,
  HSG_SWEEP_HALF = 1,         /* one launch per half-sweep */
  HSG_SWEEP_FUSED = 2,        /* one launch per sweep through shared memory (pairs of OR sweeps) */
  HSG_SWEEP_WAVE = 3,         /* one launch per sweep, odd blocks trailing even blocks in L2 */
  HSG_SWEEP_STAGED = 4        /* one launch per half-sweep, neighbour rows staged in shared memory */
};

enum {
  HSG_VARIANT_AUTO = 0,
  HSG_VARIANT_TWO_PASS = 1,   /* hsg_step replays a CUDA graph of one launch per phase */
  HSG_VARIANT_PERSISTENT = 2  /* hsg_step runs all its steps in one cooperative launch whose
                                 blocks meet at bounded grid barriers between phases */
};

/* Fill *opt with the defaults listed above. */
void hsg_default_options(hsg_options* opt);

/*
 * Create a context holding one disorder sample (Sec. 3.2: R = R_T R_O systems
 * with the same J and H).  temps: n_temps strictly increasing positive
 * temperatures (host, copied).  J, H: host arrays as described above, copied;
 * the caller keeps ownership.  Spins start uniform on the sphere from the
 * Philox init stream.  Returns HSG_EINVAL for odd L, L < 4, n_temps < 1,
 * n_replicas < 1, unsorted or non-finite temperatures, non-finite J or H.
 */
hsg_status hsg_create(hsg_ctx** out, int L, const double* temps, int n_temps, int n_replicas,
                      const float* J, const float* H, uint64_t seed, const hsg_options* opt);

/*
 * Create a context holding n_samples independent disorder samples, each with
 * its own L[s], temperatures temps[s * n_temps + t], J[s] and H[s] (H[s] or H
 * itself may be NULL).  All samples share n_temps, n_replicas, the seed and
 * the options; they are updated together by every call (Sec. 3.2, the
 * disorder average as trivial parallelism).  1 <= n_samples <= 65535, else
 * HSG_EINVAL.
 */
hsg_status hsg_create_batch(hsg_ctx** out, int n_samples, const int* L, const double* temps,
                            int n_temps, int n_replicas, const float* const* J,
                            const float* const* H, uint64_t seed, const hsg_options* opt);

/* n_steps steps of the multi-hit tile schedule, the paper's double
 * checkerboard (Sec. 3.2; Table 1, "10 x (1 HB + 10 OR)").  The lattice is cut
 * into cubic tiles of edge `tile` (4 or 8), coloured by the parity of their
 * tile coordinates.  Per step: every tile of colour 0, then every tile of
 * colour 1, gets n_rounds x (n_or OR sweeps, then n_hb HB sweeps) of its own
 * sites (even sites, then odd sites) while the rest of the lattice stays
 * fixed; then the energies (Eq. 1) and one PT pass (Eq. 4).  The k-th tile
 * sweep of a step keys its heat-bath numbers with the sample's sweep counter
 * + k; the counter advances by n_rounds (n_or + n_hb) per step.  This is a
 * different Markov chain from hsg_step's lattice sweeps (the same equilibrium
 * distribution, other autocorrelations).  HSG_EINVAL unless tile is 4 or 8,
 * every L is a multiple of 2 * tile, n_rounds >= 1 and n_or + n_hb >= 1.
 * Asynchronous. */
hsg_status hsg_step_multihit(hsg_ctx* ctx, int n_steps, int tile, int n_rounds, int n_or,
                             int n_hb);

/* n_sweeps full OR sweeps (Eq. 3), each an even then an odd half-sweep. */
hsg_status hsg_sweep_or(hsg_ctx* ctx, int n_sweeps);

/* n_sweeps full HB sweeps (Eq. 2) at each system's current temperature. */
hsg_status hsg_sweep_hb(hsg_ctx* ctx, int n_sweeps);

/* Recompute every system's energy in FP64 (Eq. 1) and run one PT pass (Eq. 4). */
hsg_status hsg_pt_exchange(hsg_ctx* ctx);

/* One PT pass with caller-supplied energies E_sys (host, double[n_samples][W],
   memory-slot order) instead of recomputed ones. */
hsg_status hsg_pt_exchange_energies(hsg_ctx* ctx, const double* E_sys);

/* n_steps steps of n_hb HB sweeps + n_or OR sweeps + energies + PT.  Two-pass
   schedule: a CUDA graph of one launch per phase, captured on the first call
   and replayed per step.  Persistent schedule (needs n_or >= 1): one
   cooperative launch for all n_steps.  Automatic: the first call times both
   schedules and several chunks-per-thread settings on the context itself
   (restoring its state afterwards) and keeps the fastest; the choice is cached
   per problem shape for the process.  All settings run the same arithmetic and
   give bit-identical results. */
hsg_status hsg_step(hsg_ctx* ctx, int n_steps);

/* FP64 energies (Eq. 1) of every system, memory-slot order, into host
   double[n_samples][W].  Synchronises. */
hsg_status hsg_energies(hsg_ctx* ctx, double* E_sys);

/* The energies the last PT pass used (or the last hsg_energies result), host
   double[n_samples][W], memory-slot order, without recomputing them.  After
   hsg_step they are the energies of the state the step ended in, summed from
   per-block partials that the last OR sweep of the step leaves behind.
   Synchronises. */
hsg_status hsg_last_energies(hsg_ctx* ctx, double* E_sys);

/* Observables, caller-owned host buffers (any pointer may be NULL to skip):
 *   E    double[n_samples][n_replicas][n_temps]   energy by temperature slot
 *   q    double[n_samples][n_temps][3][3]         q^{mu nu} of replicas 0 and 1 (Eq. 5)
 *   qk   double[n_samples][n_temps][3][3][3][2]   q^{mu nu}(k) for k = (2 pi/L) e_a,
 *                                                 a = x, y, z; [re, im]; sign e^{+i k.R}
 *   perm int32[n_samples][n_replicas][n_temps]
 * q and qk need n_replicas >= 2 (else they are left untouched).  The spins are read
 * as stored; per-thread partial sums are FP32 (a few hundred terms at most), the
 * rest FP64.  HSG_ETIMEOUT if a wait for staged spins ran out.  Synchronises. */
typedef struct {
  double* E;
  double* q;
  double* qk;
  int32_t* perm;
} hsg_obs;
hsg_status hsg_measure(hsg_ctx* ctx, hsg_obs* out);

/* Replica-pair overlaps of the current state (Sec. 2: the four-replica
 * susceptibility sums chi_1, chi_2, chi_3 and the chiral overlap).  For every
 * temperature slot t and every pair (a, b) of the first min(n_replicas, 4)
 * replicas, in the order (0,1) (0,2) (1,2) (0,3) (1,3) (2,3) (hsg_info's
 * n_overlap_pairs of them), with A, B the configurations replicas a and b hold
 * at slot t:
 *   D  double[n_samples][n_temps][n_pairs][4][2]:
 *        D_ab(k) = (1/N) sum_i (s_i^A . s_i^B) e^{+i k.R_i}
 *   C  double[n_samples][n_temps][n_pairs][3][4][2]:
 *        C_ab^alpha(k) = (1/N) sum_i kappa_i^{alpha,A} kappa_i^{alpha,B} e^{+i k.R_i}
 *        with the local chirality kappa_i^alpha = s_{i+alpha} . (s_i x s_{i-alpha}),
 *        alpha = x, y, z, periodic neighbours
 * at the modes k = 0, (2 pi/L) e_x, e_y, e_z; [re, im].  The paper's four-replica
 * sums contract the components within each site, so with replicas numbered from
 * 1: chi_1(k) = N^2 |D_12|^2, chi_2(k) = N^2 D_13 conj(D_14),
 * chi_3(k) = N^2 D_13 conj(D_24).  Caller-owned host buffers; either may be NULL
 * (not both).  HSG_EINVAL when n_replicas < 2.  The spins are read as stored;
 * per-thread partial sums are FP32 (a few hundred terms at most), the rest FP64.
 * HSG_ETIMEOUT if a wait for staged spins ran out.  Synchronises. */
hsg_status hsg_measure_overlaps(hsg_ctx* ctx, double* D, double* C);

/* Spins as FP32 (x, y, z), layout described above.  *_dev take device
   pointers of the context's device; the others host pointers.  get decodes
   the stored precision; set encodes with the context's codec. */
hsg_status hsg_get_spins(hsg_ctx* ctx, float* xyz);
hsg_status hsg_set_spins(hsg_ctx* ctx, const float* xyz);
hsg_status hsg_get_spins_dev(hsg_ctx* ctx, float* xyz_dev);
hsg_status hsg_set_spins_dev(hsg_ctx* ctx, const float* xyz_dev);

/* perm as described above, host int32[n_samples][n_replicas][n_temps]. */
hsg_status hsg_get_perm(hsg_ctx* ctx, int32_t* perm);

/* Accepted PT exchanges per pair since creation, host
   uint64[n_samples][n_replicas][n_temps - 1]; and the number of PT passes
   sample 0 has done. */
hsg_status hsg_get_pt_stats(hsg_ctx* ctx, uint64_t* accepted, uint64_t* n_calls);

/* Per-sample run lengths.  active: host uint8[n_samples], nonzero = the sample
   takes part in later hsg_step / hsg_sweep_* / hsg_pt_exchange* calls; a
   frozen sample keeps its spins, temperatures, energies and counters.  NULL
   makes every sample active (the state after creation).  Each sample's sweep
   and PT counters key its own random numbers, so a sample's chain depends
   only on how many steps it took, not on the other samples.  Synchronises. */
hsg_status hsg_set_active(hsg_ctx* ctx, const uint8_t* active);

/* Sweeps and PT passes each sample has done, host uint64[n_samples] each
   (either may be NULL).  Synchronises. */
hsg_status hsg_get_counters(hsg_ctx* ctx, uint64_t* sweeps, uint64_t* pt_passes);

/* Diagnostics of the temperature random walk (Sec. 4), since creation (or as
   restored from a checkpoint), host buffers (either may be NULL):
     moved   uint64[n_samples][n_replicas][n_temps]: PT passes after which the
             configuration that held temperature slot t before the pass holds
             another slot (p_diff(T_t) = moved / n_passes)
     tunnel  uint32[n_samples][n_replicas][n_temps] by memory slot: closed loops
             T_1 -> T_{n_temps} -> T_1 the configuration has travelled
             (tunnelling events); it starts at T_1 if it starts in slot 0
   n_passes: PT passes sample 0 has done.  Synchronises. */
hsg_status hsg_get_pt_diagnostics(hsg_ctx* ctx, uint64_t* moved, uint32_t* tunnel,
                                  uint64_t* n_passes);

/* Checkpoint and resume.  A checkpoint holds the whole state of the Markov
   chain and its statistics: the spins exactly as stored, the temperature
   permutations, inverse temperatures, last energies, sweep and PT counters,
   PT acceptance counts and diagnostics.  It can be loaded into a context
   created with the same samples (sizes, temperatures, J and H), replicas,
   precision, coupling format and seed; the chain then continues bit for bit
   as if it had not been interrupted (the step schedule does not matter).
   The blob is host memory owned by the caller; hsg_checkpoint_size gives its
   size.  Save and load synchronise.  Load returns HSG_EINVAL (and changes
   nothing) for a blob of another context, a truncated or foreign blob. */
hsg_status hsg_checkpoint_size(hsg_ctx* ctx, size_t* bytes);
hsg_status hsg_checkpoint_save(hsg_ctx* ctx, void* buf, size_t bytes);
hsg_status hsg_checkpoint_load(hsg_ctx* ctx, const void* buf, size_t bytes);

typedef struct {
  int n_samples, n_temps, n_replicas;
  int W;                   /* systems per sample */
  int Wp;                  /* systems per sample as stored (multiple of 8) */
  int precision, j_fp16, variant;
  long long total_sites;   /* sum over samples of L^3 */
  long long total_spins;   /* total_sites * W */
  long long spin_bytes;    /* device bytes of stored spins */
  long long rec_bytes;     /* device bytes of coupling/field records */
  uint64_t sweep_count;    /* sweeps sample 0 has done (hsg_get_counters: every sample) */
  uint64_t pt_count;       /* PT passes sample 0 has done */
  void* stream;            /* the cudaStream_t the context runs on */
  int chunks_per_thread;   /* sweep kernels: chunks of 4 systems one thread walks */
  int n_passes;            /* system-blocked passes per step (1: no blocking) */
  long long pass_bytes;    /* footprint bound of a pass in use (0: one pass) */
  int n_overlap_pairs;     /* replica pairs hsg_measure_overlaps reports (0 if n_replicas < 2) */
  int sweep_kernel;        /* HSG_SWEEP_HALF, HSG_SWEEP_FUSED, HSG_SWEEP_WAVE or
                              HSG_SWEEP_STAGED: the over-relaxation sweep in use */
  int fused_band_rows;     /* fused sweep: rows of y per block of sample 0 (L: whole planes) */
  int fused_items;         /* fused sweep: work items (columns of planes) per launch */
  int wave_lag;            /* wave sweep: the lag in use (even blocks) */
  int staged;              /* nonzero: the over-relaxation sweep stages its neighbour rows */
} hsg_info;
hsg_status hsg_get_info(hsg_ctx* ctx, hsg_info* info);

/*
 * FP64 energies of W systems given as caller-owned device arrays, computed
 * without allocating any device memory.  The paper has no counterpart; this
 * entry point exists for callers that must not let a library allocate: code
 * that runs while a CUDA graph is being captured (cudaMalloc is not allowed
 * there), programs whose device memory belongs to their own pool allocator,
 * and loops that cannot afford the device synchronisation cudaMalloc/cudaFree
 * can cause.
 *   spins_dev  float[W][L^3][3], (x, y, z) per site (the hsg_get_spins layout)
 *   J_dev      float[L^3][3] bonds (i, i + e_a); H_dev float[L^3][3] or NULL
 *   E_dev      double[W] output, E_w = -sum_bonds J s.s - sum_i H.s
 *   stream     cudaStream_t, NULL for the default stream; the call is
 *              asynchronous on it
 * Scratch: block partial sums go to one static __device__ array of 524288
 * doubles (4 MiB) that every GPU loading the library keeps until the process
 * exits.  Sizes with W * ceil(L^3 / 2048) > 524288 are rejected with
 * HSG_EINVAL (e.g. L = 128 allows W <= 512).  All calls share the array:
 * calls that overlap on the GPU (other streams, other host threads) race on
 * it, so serialise them.  Each call overwrites every partial it reads, so
 * nothing needs clearing between calls.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  Errors: HSG_EINVAL for bad
 * sizes or NULL pointers, HSG_ECUDA for a failed launch; the text is in
 * hsg_last_error(NULL).
 */
hsg_status hsg_energies_xyz_noalloc(const float* spins_dev, const float* J_dev,
                                    const float* H_dev, int L, int W, double* E_dev,
                                    void* stream);

/*
 * The device Philox4x32-10 generator the heat-bath sweeps use (Salmon et al.,
 * SC'11), on n host counters ctr[n][4] with key (seed & 0xffffffff, seed >> 32),
 * written to out[n][4].  For checking the device generator against other
 * implementations.  Synchronous; uses the current device.
 */
hsg_status hsg_philox(const uint32_t* ctr, long long n, uint64_t seed, uint32_t* out);

/* Wait for all work of the context; returns any pending device error. */
hsg_status hsg_sync(hsg_ctx* ctx);

/* Text of the last error on ctx (or of the last failed create if ctx is NULL). */
const char* hsg_last_error(const hsg_ctx* ctx);
const char* hsg_status_string(hsg_status st);

/* Free every resource of ctx (NULL is accepted). */
void hsg_destroy(hsg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HSG_H */
