// Over-relaxation sweeps (Sec. 3.1, Eq. 3) that stage their data instead of
// loading it into registers, and the wave launch that does both half-sweeps of
// a sweep at once.
//
// Staged block body.  A block of the sweep block table updates 256 consecutive
// storage sites of one parity: R = 256 / (L/2) whole rows y0 .. y0+R-1 of one
// plane z (L a power of 2, L >= 32).  Its sites read the opposite parity in
// rows y0-1 .. y0+R of plane z (the +-x and +-y neighbours) and in rows
// y0 .. y0+R-1 of planes z-1 and z+1.  Those rows are contiguous runs of the
// parity-split layout, so per component plane and chunk group they reach
// shared memory as six cp.async.bulk copies (the rows y0-1 and y0+R apart, as
// they wrap in y).  The block walks its chunk groups through a two-stage ring:
// while it computes chunk group g, the copies of g+1 are in flight.  Each stage
// has a full mbarrier carrying the copies' bytes; a warp that has read its
// neighbours of a stage counts itself out on the stage's counter, and the last
// warp to do so issues the copies of the stage's next chunk group, so no warp
// waits for another except through the data.  The spins a thread updates come
// by a plain load issued before its wait; the update is the per-half-sweep
// kernel's, in the same operations and order, so the results are bit for bit
// the same.  Every wait is bounded: one that runs out sets the error word, and
// the block stops computing but keeps waiting (bounded) for the copies it
// issued before it exits.
//
// Wave launch.  One launch has one block per (block table entry, parity): the
// blocks of the two per-half-sweep launches.  A block takes a ticket on entry
// (an atomic counter) and does the work the host-built order assigns to it.
// The order walks the even blocks in table order (z-major within a chunk
// group) and inserts each odd block `lag` even blocks after the last even block
// it depends on.  An odd block of planes [z0, z1] reads the even sites of
// planes z0-1 .. z1+1 (new values) and overwrites odd sites that the even
// blocks of those planes read (old values), so before its update it waits until
// every even block of those planes has signalled completion.  Those blocks hold
// earlier tickets, so they are already running and never wait themselves: no
// wait can deadlock, whatever the number of resident blocks.  Every even site
// sees only old odd spins and every odd site only new even spins, so the
// result is that of the even half-sweep followed by the odd one, bit for bit.
// Staged odd blocks read the even spins through bulk copies (L2, after a proxy
// fence); unstaged odd blocks read them bypassing L1.  Between the even update
// of a plane and the odd updates that read it lie about `lag` blocks of work,
// so the opposite parity, which two separate launches read from DRAM a second
// time, mostly comes from L2.  The last block to finish resets the ticket and
// completion counters and advances the epoch the completion flags carry, so
// each launch (and each replay of a captured graph) starts clean.
#include "hsg_async.cuh"
#include "hsg_kernels.cuh"

namespace hsg {

namespace {

constexpr int NW = SWEEP_BS / 32;   // warps per block

// Wait until *f == want, at most limit_ns.
__device__ __forceinline__ bool wait_flag(const unsigned int* f, unsigned int want,
                                          unsigned long long limit_ns) {
  const volatile unsigned int* v = f;
  if (*v == want) return true;
  const unsigned long long t0 = now_ns();
  while (*v != want) {
    if (now_ns() - t0 > limit_ns) return false;
    __nanosleep(128);
  }
  return true;
}

// Chunks of one component plane of a stage: rows [y0-1 .. y0+R] of plane z,
// then rows [y0 .. y0+R-1] of plane z-1, then of plane z+1 (R Lh = 256).
__host__ __device__ constexpr int stage_plane_chunks(int Lh) { return 3 * SWEEP_BS + 2 * Lh; }

// One block of an over-relaxation half-sweep (parity p.parity) with staged
// neighbour rows; smem: dynamic shared memory laid out as in staged_smem().
template <int F, bool J16, bool EN>
__device__ __forceinline__ void staged_block(const SweepParams& p, int bidx, unsigned char* smem) {
  constexpr int VEC = FmtInfo<F>::VEC, PL = FmtInfo<F>::PLANES, CH = FmtInfo<F>::CHUNK;
  constexpr int S = STAGED_STAGES;
  using Chunk = typename FmtInfo<F>::Chunk;
  constexpr bool MIXED = (F == FMT_F16) && J16;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  int* cnt = reinterpret_cast<int*>(smem + 64);
  float* esum = reinterpret_cast<float*>(smem + STAGED_HEAD);
  unsigned char* stages = smem + p.stage_off;

  const int4 blk = p.blocks[bidx];
  if (!p.active[blk.x]) return;   // a frozen sample (block-uniform)
  const SampleDev& sd = p.samples[blk.x];
  const int L = sd.L, Lh = sd.Lh, R = SWEEP_BS / Lh;
  const int par = p.parity;
  const uint32_t half_n = (uint32_t)sd.N >> 1;
  const int g0 = blk.y * p.GPT, g1 = min(p.G, g0 + p.GPT), ng = g1 - g0;
  const int r0 = blk.z / Lh;                  // first row (y + L z) of the block
  const int z = r0 / L, y0 = r0 - z * L;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pc = stage_plane_chunks(Lh);
  const long long gstride = (long long)sd.N * CH;
  const uint32_t tx_bytes = (uint32_t)(PL * pc * CH);

  // the copy this lane issues for a stage (lanes 0 .. 6 PL - 1 of the issuing warp)
  long long c_src = 0;
  uint32_t c_dst = 0, c_bytes = 0;
  if (lane < 6 * PL) {
    const int pl = lane / 6, kind = lane - 6 * (lane / 6);
    const uint32_t ob = (uint32_t)(1 - par) * half_n;
    int row, dst, nrows = R;
    if (kind == 0) {
      row = (y0 == 0 ? L - 1 : y0 - 1) + L * z, dst = 0, nrows = 1;
    } else if (kind == 1) {
      row = y0 + L * z, dst = Lh;
    } else if (kind == 2) {
      row = (y0 + R == L ? 0 : y0 + R) + L * z, dst = (R + 1) * Lh, nrows = 1;
    } else if (kind == 3) {
      row = y0 + L * (z == 0 ? L - 1 : z - 1), dst = (R + 2) * Lh;
    } else {
      row = y0 + L * (z + 1 == L ? 0 : z + 1), dst = (2 * R + 2) * Lh;
    }
    if (kind < 5) {
      c_src = sd.spin_off + (long long)pl * sd.plane_stride + (long long)(ob + (uint32_t)row * Lh) * CH;
      c_dst = (uint32_t)((pl * pc + dst) * CH);
      c_bytes = (uint32_t)(nrows * Lh * CH);
      // HSG_CHECK builds: the rows within the opposite half, the copy within its
      // stage (else copy the same number of bytes from the plane's start: the
      // stage's byte count still completes, the results are flagged)
      if (HSG_OUT_OF_BOUNDS(row >= 0 && (long long)(row + nrows) * Lh <= (long long)half_n &&
                                c_dst + c_bytes <= (uint32_t)p.stage_bytes,
                            p.bounds_err))
        c_src = sd.spin_off + (long long)pl * sd.plane_stride;
    }
  }
  auto issue = [&](int i) {   // the copies of chunk group g0 + i into stage i % S (one warp)
    const int s = i % S;
    if (lane == 0) mbar_expect_tx(&full[s], tx_bytes);
    __syncwarp();
    if (c_bytes)
      bulk_copy_g2s(stages + s * p.stage_bytes + c_dst, p.spins + c_src + (long long)(g0 + i) * gstride,
                    c_bytes, &full[s]);
  };
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      cnt[s] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0) {
    for (int i = 0; i < S && i < ng; ++i) issue(i);
  }

  // this thread's site, its neighbours' chunk offsets in a stage plane (+x, -x,
  // +y, -y, +z, -z) and its couplings
  const int lr = tid / Lh, hx = tid - lr * Lh;
  const int y = y0 + lr;
  const int x = 2 * hx + ((par + y + z) & 1);
  const int xp = (x + 1 == L) ? 0 : x + 1, xm = (x == 0) ? L - 1 : x - 1;
  int off[6];
  off[0] = (lr + 1) * Lh + (xp >> 1);
  off[1] = (lr + 1) * Lh + (xm >> 1);
  off[2] = (lr + 2) * Lh + hx;
  off[3] = lr * Lh + hx;
  off[4] = (2 * R + 2) * Lh + lr * Lh + hx;
  off[5] = (R + 2) * Lh + lr * Lh + hx;
  uint32_t own = (uint32_t)par * half_n + (uint32_t)blk.z + (uint32_t)tid;
  bool store_ok = true;
  {
    // HSG_CHECK builds: the site in this parity's half and its neighbours within
    // the stage plane (else read in-bounds slots and write nothing back)
    bool bad = HSG_OUT_OF_BOUNDS((uint32_t)blk.z + (uint32_t)tid < half_n, p.bounds_err);
#pragma unroll
    for (int n = 0; n < 6; ++n) bad = bad || HSG_OUT_OF_BOUNDS(off[n] >= 0 && off[n] < pc, p.bounds_err);
    if (bad) {
      own = (uint32_t)par * half_n;
#pragma unroll
      for (int n = 0; n < 6; ++n) off[n] = 0;
      store_ok = false;
    }
  }
  float j6[6], h3[3];
  uint32_t jh[6];
  load_record<J16>(p.rec, sd.rec_off + own, j6, h3);
  if (MIXED) load_record_j16(p.rec, sd.rec_off + own, jh);
  unsigned char* own_base = p.spins + sd.spin_off + (long long)own * CH;
  const long long ps = sd.plane_stride;

  bool ok = true;
  int i = 0;
  for (; i < ng; ++i) {
    const int s = i % S;
    const uint32_t ph = (uint32_t)(i / S) & 1u;
    unsigned char* own_p = own_base + (long long)(g0 + i) * gstride;
    Chunk c[PL];
    load_chunks<F, LD_PLAIN>(own_p, ps, c);
    float e[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) e[v] = 0.0f;
    if (!__all_sync(0xffffffffu, mbar_wait(&full[s], ph, p.timeout_ns))) {
      ok = false;
      break;
    }
    const unsigned char* st = stages + s * p.stage_bytes;
    Chunk nc[6][PL];
#pragma unroll
    for (int n = 0; n < 6; ++n)
#pragma unroll
      for (int pl = 0; pl < PL; ++pl)
        nc[n][pl] = *reinterpret_cast<const Chunk*>(st + (pl * pc + off[n]) * CH);

    // local field h = sum_n J_n s_n + H, in the order +x, -x, +y, -y, +z, -z
    Spins<VEC> hf;
    if constexpr (MIXED) {
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
    // every neighbour value is in registers: count this warp out of the stage;
    // the last warp refills it with the chunk group S further on
    {
      int last = 0;
      __syncwarp();
      if (lane == 0) {
        last = atomicAdd(&cnt[s], 1) == NW - 1;
        if (last) atomicExch(&cnt[s], 0);
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      if (last && i + S < ng) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(i + S);
      }
    }
    {
      const float2 hx2 = f2(h3[0]), hy2 = f2(h3[1]), hz2 = f2(h3[2]);
#pragma unroll
      for (int k = 0; k < VEC / 2; ++k) {
        hf.x[k] = add2(hf.x[k], hx2);
        hf.y[k] = add2(hf.y[k], hy2);
        hf.z[k] = add2(hf.z[k], hz2);
      }
    }
    Spins<VEC> sv;
    decode<F>(c, sv);
#pragma unroll
    for (int k = 0; k < VEC / 2; ++k) or_move2(sv.x[k], sv.y[k], sv.z[k], hf.x[k], hf.y[k], hf.z[k]);
    encode<F>(sv, c);
    if (store_ok) store_chunks<F>(own_p, ps, c);
    if constexpr (EN) {
      // energy of the new state from the stored values: every bond joins one
      // odd and one even site, E = - sum_odd s_i.h_i - sum_even H_j.s_j
      Spins<VEC> stv;
      decode<F>(c, stv);
#pragma unroll
      for (int k = 0; k < VEC / 2; ++k) {
        float2 d;
        if (par == 1) {
          d = dot3_2(stv.x[k], stv.y[k], stv.z[k], hf.x[k], hf.y[k], hf.z[k]);
        } else {
          d = dot3_2(stv.x[k], stv.y[k], stv.z[k], f2(h3[0]), f2(h3[1]), f2(h3[2]));
        }
        e[2 * k] = -d.x;
        e[2 * k + 1] = -d.y;
      }
      static_assert(VEC == 4, "the scattered warp sum takes four systems per chunk");
      const float t = warp_sum4_scatter(e, lane);
      if ((lane & 7) == 0) esum[warp * p.GPT * VEC + i * VEC + (lane >> 3)] = t;
    }
  }
  if (!ok) {
    // a wait ran out: flag it and give the copies in flight a bounded time to
    // land before the block's shared memory is released
    if (lane == 0) atomicExch(p.err, 1u);
    for (int q = i; q < ng && q < i + S; ++q)
      mbar_wait(&full[q % S], (uint32_t)(q / S) & 1u, p.timeout_ns);
  }
  if constexpr (EN) {
    __syncthreads();
    double* out = p.epart + ((long long)par * p.n_blocks + bidx) * p.Wp;
    for (int j = tid; j < p.Wp; j += SWEEP_BS) {
      double acc = 0.0;
      const int jj = j - g0 * VEC;
      if (jj >= 0 && jj < ng * VEC) {
        for (int w = 0; w < NW; ++w) acc += (double)esum[w * p.GPT * VEC + jj];
      }
      out[j] = acc;
    }
  }
  __syncthreads();   // the ring and its barriers are reused by nothing after this
}

template <int F, bool J16, bool EN>
__global__ void __launch_bounds__(SWEEP_BS, 4) k_staged_half(const SweepParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int k = p.reverse ? p.n_launch - 1 - (int)blockIdx.x : (int)blockIdx.x;
  staged_block<F, J16, EN>(p, p.blk_base + k, smem);
}

template <int F, bool J16, bool EN, bool STG>
__global__ void __launch_bounds__(SWEEP_BS, 4) k_wave_sweep(const WaveParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ unsigned int s_ticket, s_epoch;
  if (threadIdx.x == 0) {
    s_ticket = atomicAdd(P.state, 1u);
    s_epoch = *(volatile unsigned int*)(P.state + 2);
  }
  __syncthreads();
  const unsigned int want = s_epoch + 1u;
  // (a ticket beyond the launch would mean counters left inconsistent: no work)
  const bool valid = s_ticket < (unsigned int)P.n_tickets;
  const int code = valid ? P.order[P.t0 + (int)s_ticket] : 0;
  const int b = code >> 1, parity = valid ? (code & 1) : 2;
  SweepParams sp = P.sw;
  sp.parity = parity & 1;
  if (!valid) {
    if (threadIdx.x == 0) atomicExch(P.err, 1u);
  } else if (parity == 0) {
    if constexpr (STG) staged_block<F, J16, EN>(sp, b, smem);
    else sweep_block<F, false, J16, false, EN, false>(sp, b, reinterpret_cast<float*>(smem));
  } else {
    // every even block of the planes this block reads or overwrites
    const int4 d = P.deps[b];
    bool late = false;
    for (int i = d.x + (int)threadIdx.x; i < d.y; i += SWEEP_BS)
      late |= !wait_flag(P.flags + i, want, P.timeout_ns);
    for (int i = d.z + (int)threadIdx.x; i < d.w; i += SWEEP_BS)
      late |= !wait_flag(P.flags + i, want, P.timeout_ns);
    if (b == P.inject_block && threadIdx.x == 0) late |= !wait_flag(P.flags + P.never, want, P.timeout_ns);
    __threadfence();
    if (STG) asm volatile("fence.proxy.async.global;" ::: "memory");
    if (__syncthreads_or(late)) {
      if (threadIdx.x == 0) atomicExch(P.err, 1u);
    } else {
      if constexpr (STG) staged_block<F, J16, EN>(sp, b, smem);
      else sweep_block<F, false, J16, false, EN, true>(sp, b, reinterpret_cast<float*>(smem));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (parity == 0) atomicExch(P.flags + b, want);
    if (atomicAdd(P.state + 1, 1u) == (unsigned int)P.n_tickets - 1u) {
      // every block has finished: reset for the next launch
      atomicExch(P.state, 0u);
      atomicExch(P.state + 1, 0u);
      atomicAdd(P.state + 2, 1u);
      __threadfence();
    }
  }
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int F, bool J16, bool EN, bool STG>
cudaError_t launch_w(const WaveParams& p, size_t smem, cudaStream_t st) {
  cudaError_t e = allow_smem(k_wave_sweep<F, J16, EN, STG>, smem);
  if (e != cudaSuccess) return e;
  k_wave_sweep<F, J16, EN, STG><<<p.n_tickets, SWEEP_BS, smem, st>>>(p);
  return cudaGetLastError();
}

template <int F>
cudaError_t launch_wf(bool j16, bool en, bool stg, const WaveParams& p, size_t smem, cudaStream_t st) {
  if (stg) {
    if (j16) return en ? launch_w<F, true, true, true>(p, smem, st) : launch_w<F, true, false, true>(p, smem, st);
    return en ? launch_w<F, false, true, true>(p, smem, st) : launch_w<F, false, false, true>(p, smem, st);
  }
  if (j16) return en ? launch_w<F, true, true, false>(p, smem, st) : launch_w<F, true, false, false>(p, smem, st);
  return en ? launch_w<F, false, true, false>(p, smem, st) : launch_w<F, false, false, false>(p, smem, st);
}

template <int F, bool J16, bool EN>
cudaError_t launch_h(const SweepParams& p, int n_blocks, size_t smem, cudaStream_t st) {
  cudaError_t e = allow_smem(k_staged_half<F, J16, EN>, smem);
  if (e != cudaSuccess) return e;
  k_staged_half<F, J16, EN><<<n_blocks, SWEEP_BS, smem, st>>>(p);
  return cudaGetLastError();
}

template <int F>
cudaError_t launch_hf(bool j16, bool en, const SweepParams& p, int n_blocks, size_t smem,
                      cudaStream_t st) {
  if (j16) return en ? launch_h<F, true, true>(p, n_blocks, smem, st) : launch_h<F, true, false>(p, n_blocks, smem, st);
  return en ? launch_h<F, false, true>(p, n_blocks, smem, st) : launch_h<F, false, false>(p, n_blocks, smem, st);
}

template <int F>
cudaError_t occupancy_f(bool j16, bool stg, size_t smem, int* blocks_per_sm) {
  const void* fn = stg ? (j16 ? (const void*)k_wave_sweep<F, true, false, true>
                              : (const void*)k_wave_sweep<F, false, false, true>)
                       : (j16 ? (const void*)k_wave_sweep<F, true, false, false>
                              : (const void*)k_wave_sweep<F, false, false, false>);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, SWEEP_BS, smem);
}

}  // namespace

bool fmt_has_wave(int fmt) { return fmt == FMT_F32 || fmt == FMT_F16 || fmt == FMT_BF16; }

bool lattice_has_staged(int L) { return L >= 32 && (L & (L - 1)) == 0; }

int staged_stage_bytes(int fmt, int Lh_max) {
  const int ch = fmt == FMT_F32 ? 16 : 8;   // component formats: 3 planes
  return 3 * stage_plane_chunks(Lh_max) * ch;
}

// [0, STAGED_HEAD): mbarriers and stage counters; then the energy sums of the
// warps (energy sweeps); then, 128-byte aligned, the ring of stages.
size_t staged_smem(int fmt, int gpt, bool energy, int Lh_max, int* stage_off) {
  const size_t esum = energy ? sizeof(float) * NW * (size_t)gpt * 4 : 0;
  const size_t off = (STAGED_HEAD + esum + 127) / 128 * 128;
  *stage_off = (int)off;
  return off + (size_t)STAGED_STAGES * staged_stage_bytes(fmt, Lh_max);
}

cudaError_t wave_occupancy(int fmt, bool j16, bool staged, size_t smem, int* blocks_per_sm) {
  switch (fmt) {
    case FMT_F32: return occupancy_f<FMT_F32>(j16, staged, smem, blocks_per_sm);
    case FMT_F16: return occupancy_f<FMT_F16>(j16, staged, smem, blocks_per_sm);
    case FMT_BF16: return occupancy_f<FMT_BF16>(j16, staged, smem, blocks_per_sm);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_wave(int fmt, bool j16, bool energy, bool staged, const WaveParams& p, size_t smem,
                        cudaStream_t st) {
  if (p.n_tickets <= 0) return cudaSuccess;
  switch (fmt) {
    case FMT_F32: return launch_wf<FMT_F32>(j16, energy, staged, p, smem, st);
    case FMT_F16: return launch_wf<FMT_F16>(j16, energy, staged, p, smem, st);
    case FMT_BF16: return launch_wf<FMT_BF16>(j16, energy, staged, p, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_staged_half(int fmt, bool j16, bool energy, const SweepParams& p, int n_blocks,
                               size_t smem, cudaStream_t st) {
  if (n_blocks <= 0) return cudaSuccess;
  switch (fmt) {
    case FMT_F32: return launch_hf<FMT_F32>(j16, energy, p, n_blocks, smem, st);
    case FMT_F16: return launch_hf<FMT_F16>(j16, energy, p, n_blocks, smem, st);
    case FMT_BF16: return launch_hf<FMT_BF16>(j16, energy, p, n_blocks, smem, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hsg
