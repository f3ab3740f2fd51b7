// Triple products over cells on the 5th-generation tensor cores (tcgen05, TMEM accumulators).
//
// The contraction of Eq. bi_sco / Eq. new_bispec in real space,
//     T[f, (i, j), c] = sum_x A_{f,i}(x) B_{f,j}(x) C_c(x),
// is a GEMM over the cells x whose two sides are chosen per launch by the host (plan_triple_tc):
// of the three staged fields of an output, two form a product row U_r = S_u S_v (the M side, at
// most 3 x 128 rows per CTA) and the third is a single-field column W_w (the N side).  The choice
// that needs the fewest product rows wins: for B_0, B_2, B_000, B_202 the rows are the symmetric
// products F_0,j F_0,k and F_0,j G (228 rows for 19 bins) and the columns are F_0,i and F_2,i
// (38), instead of 380 rows F_l,i F_0,j against 21 columns.
//
// Precision: every operand is split into f16 hi + lo (about 22 significant bits, like a tf32
// split) after an exact power-of-two scale taken from the largest |value| of each staged field
// (recorded by the last shell pass), so that no product row exceeds 2^14 and no column 2^14 in
// magnitude.  The N side holds hi and lo of every column interleaved (rows 2w and 2w + 1 of the
// operand), so two products per 16-cell k step and row tile, U_hi x [W_hi W_lo] and
// U_lo x [W_hi W_lo], give all four terms of (U_hi + U_lo)(W_hi + W_lo): tcgen05.mma kind::f16,
// M = 128, N = 2 x columns rounded up to 16, K = 16, FP32 accumulation in tensor memory.  One
// instruction of N <= 64 costs the same as one of N = 16 on this part, so the column side is
// packed as wide as the launch allows.
//
// Per CTA:
//   * one loader thread copies the staged fields of each chunk of 128 cells with bulk asynchronous
//     copies (the TMA unit) into a ring of two or three shared-memory buffers: the float shell
//     fields are stored chunk-interleaved (all fields' rows of a chunk follow each other), so every
//     run of consecutive field indices is one copy; completion on an mbarrier with a transaction
//     count, and the consumers free a buffer on a second mbarrier when they are done with it;
//   * two producer threads per product row (each on half of the 16-cell k steps of a 64-cell stage)
//     form U = S_u S_v scale, split it into f16 hi and lo and write both into tensor memory
//     (tcgen05.st): the M-side operand never passes through shared memory;
//   * four warps write the N-side operand (hi and lo of every column) into shared memory in the
//     canonical K-major layout without swizzle (8 rows x 16-byte core matrices, one 16-byte row
//     store per column, half and 8-cell group);
//   * one thread issues the products of each stage and commits the stage to an mbarrier that frees
//     its tensor-memory and shared-memory slots (a ring of two to four stages, as tensor memory allows);
//   * every FLUSH stages (4096 cells) the producers read the accumulators back (tcgen05.ld), add
//     the hi and lo columns and add the result into compensated float32 sums in shared memory (the
//     scales are constant within the CTA, so the sums stay scaled);
//   * at the end the CTA undoes the scales in float64 and writes every requested output as
//     part[cta][row][col] through the plan's gather table, reduced in a fixed order by the same
//     kernels as the other paths.
// Every wait is bounded (clock64 against `limit`); on expiry the kernel records NPC_ERR_TIMEOUT in
// the device status word, the other roles leave their loops, the control and loader threads wait
// (with a fixed bound) for their products and copies in flight, and the allocating warp frees
// tensor memory.  A staged field whose largest |value| lies outside [2^-57, 2^63) (other than an
// all-zero field) records NPC_ERR_NUMERIC: the scaled split would lose precision or overflow.
#pragma once

#include <cstdint>

namespace tc {

constexpr int CHUNK = 128;        // cells per bulk-copy chunk (512 bytes per staged field)
constexpr int SROW = CHUNK;       // floats between staged field rows (a row is rotated by rf_rot of
                                  // its field: 16-byte reads of eight fields hit distinct banks)
// 64-cell stages, two in flight (the most tensor memory holds beside two 128-row accumulator tiles
// of N = 80): a stage costs about 1,300 cycles of hand-over besides its work, so 32-cell stages with
// four in flight measured 0.44-0.47 ms at 256^3 against 0.33 ms; one producer thread per row
// instead of two measured 0.38 ms
constexpr int AST = 64;           // cells per stage: k steps of 16, half of them per producer thread
constexpr int KSTEPS = AST / 16;
constexpr int PPR = 2;            // producer threads per product row
constexpr int KPT = KSTEPS / PPR; // k steps per producer thread
constexpr int PWT = 4 * PPR;      // producer warps per 128-row tile
constexpr int SPC = CHUNK / AST;  // stages per chunk
constexpr int NSA_MAX = 4;        // stages in flight at most (tensor-memory and operand rings)
constexpr int FLUSH = 4096 / AST; // stages between float64 flushes (4096 cells)
constexpr int NBW = 4;            // warps writing the N-side operand
constexpr int MAXN = 128;         // largest N (64 single-field columns, hi and lo)
constexpr int ACOLS = KSTEPS * 16;// tensor-memory columns of one stage and row tile (hi 8 + lo 8 per k step)
constexpr int MAX_SLOTS = 96;     // staged fields per launch at most
constexpr int EMIN = -56, EMAX = 63;   // admissible binary exponents of a field's largest |value|
                                       // (|S_u S_v| < 2^126 stays finite in float)
constexpr long long DRAIN_LIMIT = 1ll << 31;  // cycles a clean-up wait may take
static_assert(CHUNK == RCH && SROW == RCH, "a chunk buffer row is one row of the chunk-interleaved fields");

// The launch's orientation, built on the host (plan_triple_tc) and kept in device tables.
// Staged slots are numbered by increasing field index, so that a run of consecutive fields is one
// contiguous block of every chunk.
struct Plan {
  int nmrow;             // product rows U_r = S_rx[r] S_ry[r]
  int nmcol;             // single-field columns W_w = S_cz[w]
  int n;                 // MMA N: 2 nmcol rounded up to 16
  int nsa;               // stages in flight
  int nout;              // outputs: rows x columns of the part layout
  int nstage;            // staged fields
  int nrun;              // runs of consecutive field indices among them
  int nfield;            // fields of the shell-field array (its chunk stride)
  const int16_t* rx;     // [nmrow] staged slots of the two factors
  const int16_t* ry;
  const int16_t* cz;     // [nmcol] staged slot of each column
  const int* sfield;     // [nstage] field index of each staged slot (increasing)
  const int* runs;       // [nrun][2] first slot and length of each run
  const int* gidx;       // [nout] product row * nmcol + column of each output, or -1 (a zero column)
};

// tensor memory: accumulators of row tile t at columns [t n, (t + 1) n); the M-side ring after them
__host__ __device__ constexpr int a_col(int n, int nt, int slot, int t, int j) {
  return nt * n + ((slot * nt + t) * KSTEPS + j) * 16;
}
__host__ __device__ constexpr uint32_t tmem_cols_for(int n, int nt, int nsa) {
  return (nt * n + nsa * nt * ACOLS) <= 256 ? 256u : 512u;
}

// instruction descriptor: D f32, A and B f16, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t idesc_f16(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// try_wait may suspend the thread for a while (until the phase completes or a system time limit);
// test_wait returns at once
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_poll(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of parity `parity`.  Gives up (false) when another role has aborted
// or after `limit` cycles, in which case it records the timeout and raises the CTA's abort flag.
// The bound is checked before every suspending probe, so that a bound shorter than the wait gives
// up even when one probe alone would have outlasted it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit, volatile int* abort,
                                          int* status) {
  if (mbar_poll(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (*abort) return false;
    if (clock64() - t0 > limit) {
      *abort = 1;
      atomicCAS(status, 0, (int)NPC_ERR_TIMEOUT);
      return false;
    }
    if (mbar_test(bar, parity)) return true;
  }
}

// The same wait taken by every lane of a warp, with one outcome for the warp: the warp goes on to
// warp-wide (.sync.aligned) tensor-memory instructions only if every lane saw the phase complete.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, long long limit, volatile int* abort,
                                          int* status) {
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, limit, abort, status));
}

// clean-up wait: fixed bound, no abort check
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > DRAIN_LIMIT) return;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// TMEM stores read their registers at issue; completion (tcgen05.wait::st) is awaited before the
// thread synchronisation that hands the stage to the MMA thread.  No memory clobber: tensor memory
// is not addressable memory, and ordinary loads may move across the store.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]));
}

// 8 columns of this warp's 32 lanes, with the wait in the same statement so that no use of the
// registers can be scheduled before the data has arrived
__device__ __forceinline__ void tmem_ld8_wait(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
      : "r"(taddr)
      : "memory");
}

// shared-memory matrix descriptor, canonical K-major layout without swizzle: core matrices of
// 8 rows x 16 bytes (rows 16 bytes apart), `lbo` bytes between core matrices along K, `sbo` bytes
// between 8-row groups along M/N; bit 46 is the descriptor version of this architecture.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(
          d),
      "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Two cells (v0 the even k element, v1 the odd one) as f16 hi and lo pairs: hi = v with the 13 low
// mantissa bits cleared (11 significant bits, exact in f16 within its normal range), lo = v - hi
// (exact in float) rounded to f16; about 22 significant bits in all.  The even element sits in the
// low half of each word.
__device__ __forceinline__ void split_f16x2(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const float h0 = __uint_as_float(__float_as_uint(v0) & 0xffffe000u);
  const float h1 = __uint_as_float(__float_as_uint(v1) & 0xffffe000u);
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(h1), "f"(h0));
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(v1 - h1), "f"(v0 - h0));
}

__device__ __forceinline__ float exp2f_int(int e) { return __int_as_float((127 + e) << 23); }      // e in [-126, 127]
__device__ __forceinline__ double exp2d_int(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// Position in a ring of `n` slots and the parity of the slot's current use (slot = i mod n,
// parity = (i / n) mod 2 for the i-th use), advanced without divisions.
struct Ring {
  int slot = 0;
  uint32_t par = 0;
  __device__ __forceinline__ void next(int n) {
    if (++slot == n) {
      slot = 0;
      par ^= 1u;
    }
  }
};

struct Smem {
  uint64_t full_tma[3];       // chunk buffer filled (transaction count)
  uint64_t chunk_free[3];     // chunk buffer read by every producer and operand warp
  uint64_t full_a[NSA_MAX];   // stage written by every producer and operand warp
  uint64_t empty_a[NSA_MAX];  // products of a stage complete (tcgen05.commit)
  uint64_t drain;             // clean-up commit
  uint32_t tmem_base;
  int abort;
};

// compensated float32 accumulation (Kahan): s + c carries the sum to about twice float precision
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// dynamic shared memory of k_triple_tc<nt> and its carve-up
struct Layout {
  size_t buf, btile, sums, comp, row_e, slot_e, smem, total;
};
__host__ __device__ inline Layout tc_layout(int nstage, int nbuf, int nt, int n, int nmcol, int nsa) {
  Layout L{};
  L.buf = 0;
  L.btile = (((size_t)nbuf * nstage * SROW * sizeof(float)) + 1023) & ~(size_t)1023;
  L.sums = L.btile + (size_t)nsa * KSTEPS * n * 32;
  L.comp = L.sums + sizeof(float) * (size_t)nmcol * nt * 128;
  L.row_e = L.comp + sizeof(float) * (size_t)nmcol * nt * 128;
  L.slot_e = L.row_e + sizeof(int) * (size_t)nt * 128;
  L.smem = L.slot_e + sizeof(int) * (MAX_SLOTS + 128);
  L.total = L.smem + sizeof(Smem);
  return L;
}

}  // namespace tc

// grid = (CTAs over the cells, groups of NT x 128 product rows); block = NT x 128 x PPR producers
// (warp PWT t + 4h + q serves tile t, lanes 32q.. of tensor memory, k steps KPT h.. of each stage)
// + NBW operand warps + the MMA warp + the loader warp.  Requires ncell % 128 == 0; R in the
// chunk-interleaved float layout (rf_index: 128-float rows, rotated by rf_rot); nbuf = 2 or 3 buffers; dynamic shared
// memory = tc_layout(...).total; fmax[f] = bits of max |R_f| (non-negative floats compare as
// unsigned integers).
template <int NT>
__global__ void __launch_bounds__(NT * 128 * tc::PPR + (tc::NBW + 2) * 32, 1)
k_triple_tc(const float* __restrict__ R, int64_t ncell, const __grid_constant__ tc::Plan P,
            const unsigned* __restrict__ fmax, double* __restrict__ part, int* status, long long limit, int nbuf) {
  using namespace tc;
  extern __shared__ __align__(16) unsigned char smem_raw[];   // descriptors and bulk copies need 16 bytes
  const int N = P.n, NSA = P.nsa, NTR = NT * 128;
  const Layout L = tc_layout(P.nstage, nbuf, NT, N, P.nmcol, NSA);
  float* buf = reinterpret_cast<float*>(smem_raw + L.buf);        // [nbuf][nstage][SROW]
  unsigned char* btile = smem_raw + L.btile;                      // [NSA][KSTEPS][N rows x 32 B]
  float* sums = reinterpret_cast<float*>(smem_raw + L.sums);      // [nmcol][NTR], scaled
  float* comp = reinterpret_cast<float*>(smem_raw + L.comp);      // their compensations
  int* row_e = reinterpret_cast<int*>(smem_raw + L.row_e);        // [NTR] exponent sums of the rows
  int* slot_e = reinterpret_cast<int*>(smem_raw + L.slot_e);      // [MAX_SLOTS] exponents, [64] column exponents,
  int* col_e = slot_e + MAX_SLOTS;                                // [64] column slots
  int* col_s = col_e + 64;
  Smem* sm = reinterpret_cast<Smem*>(smem_raw + L.smem);
  volatile int* abort = &sm->abort;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bw0 = NT * PWT;        // first operand warp
  const int mw = bw0 + NBW;        // MMA warp (allocates tensor memory)
  const int lw = mw + 1;           // loader warp
  const int nconsumer = NT * PWT + NBW;
  const uint32_t NCOLS = tmem_cols_for(N, NT, NSA);

  // cell range of this CTA, in whole chunks
  const int64_t nchunk_all = ncell / CHUNK;
  const int64_t per = (nchunk_all + gridDim.x - 1) / gridDim.x;
  const int64_t c_beg = min((int64_t)blockIdx.x * per, nchunk_all);
  const int64_t c_end = min(c_beg + per, nchunk_all);
  const int nchunk = (int)(c_end - c_beg);
  const int nst = nchunk * SPC;

  for (int i = tid; i < P.nmcol * NTR; i += blockDim.x) sums[i] = comp[i] = 0.f;
  for (int i = tid; i < NSA * KSTEPS * N * 8; i += blockDim.x) reinterpret_cast<uint32_t*>(btile)[i] = 0u;
  // binary exponent E of each staged field's largest |value| (|v| < 2^E); all-zero fields take EMIN
  for (int s = tid; s < P.nstage; s += blockDim.x) {
    const unsigned u = fmax[P.sfield[s]];
    int e = EMIN;
    if (u != 0u) {
      e = (int)((u >> 23) & 0xffu) - 126;
      if (e < EMIN || e > EMAX) {
        atomicCAS(status, 0, (int)NPC_ERR_NUMERIC);
        e = e < EMIN ? EMIN : EMAX;
      }
    }
    slot_e[s] = e;
  }
  if (warp == mw) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm->tmem_base)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    if (lane == 0) {
      for (int b = 0; b < nbuf; ++b) {
        mbar_init(&sm->full_tma[b], 1);
        mbar_init(&sm->chunk_free[b], nconsumer);
      }
      for (int b = 0; b < NSA; ++b) {
        mbar_init(&sm->full_a[b], nconsumer);
        mbar_init(&sm->empty_a[b], 1);
      }
      mbar_init(&sm->drain, 1);
      sm->abort = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
  }
  __syncthreads();
  for (int w = tid; w < P.nmcol; w += blockDim.x) {
    col_s[w] = P.cz[w];
    col_e[w] = slot_e[P.cz[w]];
  }
  fence_async_smem();   // the zeroed operand padding is read by the tensor cores
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = sm->tmem_base;

  if (warp == lw) {
    // ---- loader thread: every run of consecutive fields of a chunk is one bulk copy ----
    if (lane == 0) {
      const uint32_t bytes = (uint32_t)(P.nstage * RCH * sizeof(float));
      int issued = 0;
      Ring bf;
      for (int c = 0; c < nchunk; ++c, bf.next(nbuf)) {
        const int b = bf.slot;
        if (c >= nbuf && !mbar_wait(&sm->chunk_free[b], bf.par ^ 1u, limit, abort, status)) break;
        mbar_arrive_tx(&sm->full_tma[b], bytes);
        const size_t gchunk = (size_t)(c_beg + c);
        for (int r = 0; r < P.nrun; ++r) {
          const int s0 = P.runs[2 * r], len = P.runs[2 * r + 1];
          bulk_g2s(buf + ((size_t)b * P.nstage + s0) * SROW, R + (gchunk * P.nfield + P.sfield[s0]) * RCH,
                   (uint32_t)(len * RCH * sizeof(float)), &sm->full_tma[b]);
        }
        issued = c + 1;
      }
      // after an abort, copies nobody waited for must land before the block exits
      if (*abort)
        for (int c = max(0, issued - nbuf); c < issued; ++c) mbar_drain(&sm->full_tma[c % nbuf], (uint32_t)((c / nbuf) & 1));
    }
    __syncwarp();
  } else if (warp == mw) {
    // ---- MMA thread: the tensor-core products of every stage ----
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(N);
      const uint64_t bd0 = sdesc(smem_u32(btile), 128, 256);
      const uint32_t bstep = (uint32_t)(N * 32) >> 4;   // one k step of the operand, in descriptor units
      Ring st;
      for (int s = 0; s < nst; ++s, st.next(NSA)) {
        const int slot = st.slot;
        if (!mbar_wait(&sm->full_a[slot], st.par, limit, abort, status)) break;
        tc_fence_after();
        const bool fresh = (s % FLUSH) == 0;
#pragma unroll
        for (int j = 0; j < KSTEPS; ++j) {
          const uint64_t bd = bd0 + (uint64_t)((slot * KSTEPS + j) * bstep);
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            const uint32_t d = tbase + (uint32_t)(t * N);
            const uint32_t ahi = tbase + (uint32_t)a_col(N, NT, slot, t, j);
            mma_f16(d, ahi, bd, idesc, (fresh && j == 0) ? 0u : 1u);
            mma_f16(d, ahi + 8, bd, idesc, 1u);
          }
        }
        mma_commit(&sm->empty_a[slot]);
      }
      // every product issued must finish before tensor memory is freed
      mma_commit(&sm->drain);
      mbar_drain(&sm->drain, 0);
    }
    __syncwarp();
  } else if (warp >= bw0) {
    // ---- operand warps: hi and lo of every column, interleaved (rows 2w, 2w + 1 of the N side);
    //      unit u = (column w, 8-cell group g of the stage): one 16-byte row of hi and one of lo.
    //      A row's bank group is its index mod 8 (every other stride of the layout is a multiple of
    //      128 bytes), so lanes 2i and 2i + 1 take the same column (groups 2q, 2q + 1), a quarter
    //      warp four consecutive columns, and the odd lane of a pair stores its lo row first: the
    //      eight rows of each store fall on eight bank groups ----
    const int tb = tid - bw0 * 32;
    constexpr int GPS = AST / 8;                      // 8-cell groups per stage
    const int nunit = P.nmcol * GPS;
    constexpr int UPT = (MAXN / 2 * GPS + NBW * 32 - 1) / (NBW * 32);   // units per thread at most
    int srow[UPT], scell[UPT], d1[UPT], d2[UPT];
    float fsc[UPT];
    const bool lo_first = (tb & 1) != 0;
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
      const int u = tb + k * NBW * 32;
      const int pr = u >> 1;
      const int w = pr % P.nmcol, g = 2 * (pr / P.nmcol) + (u & 1), j = g >> 1, kh = g & 1;
      srow[k] = u < nunit ? col_s[w] * SROW : 0;
      scell[k] = 8 * g + (u < nunit ? rf_rot(P.sfield[col_s[w]]) : 0);   // rotated cell of the unit's first cell
      fsc[k] = u < nunit ? exp2f_int(14 - col_e[w]) : 0.f;
      const int dhi = j * N * 32 + ((2 * w) >> 3) * 256 + kh * 128 + ((2 * w) & 7) * 16;
      const int dlo = j * N * 32 + ((2 * w + 1) >> 3) * 256 + kh * 128 + ((2 * w + 1) & 7) * 16;
      d1[k] = lo_first ? dlo : dhi;
      d2[k] = lo_first ? dhi : dlo;
    }
    Ring st, bf;   // stage slot; chunk buffer (advanced after the chunk's last stage)
    for (int s = 0; s < nst; ++s, st.next(NSA)) {
      const int slot = st.slot;
      const int o = (s % SPC) * AST;
      const int b = bf.slot;
      if ((s % SPC) == 0 && !warp_wait(&sm->full_tma[b], bf.par, limit, abort, status)) break;
      if (s >= NSA && !warp_wait(&sm->empty_a[slot], st.par ^ 1u, limit, abort, status)) break;
      const float* stage = buf + (size_t)b * P.nstage * SROW;
      unsigned char* bslot = btile + (size_t)slot * KSTEPS * N * 32;
#pragma unroll
      for (int k = 0; k < UPT; ++k) {
        if (tb + k * NBW * 32 < nunit) {
          const float4 a0 = *reinterpret_cast<const float4*>(stage + srow[k] + ((o + scell[k]) & (CHUNK - 1)));
          const float4 a1 = *reinterpret_cast<const float4*>(stage + srow[k] + ((o + scell[k] + 4) & (CHUNK - 1)));
          const float f = fsc[k];
          uint4 hi, lo;
          split_f16x2(a0.x * f, a0.y * f, hi.x, lo.x);
          split_f16x2(a0.z * f, a0.w * f, hi.y, lo.y);
          split_f16x2(a1.x * f, a1.y * f, hi.z, lo.z);
          split_f16x2(a1.z * f, a1.w * f, hi.w, lo.w);
          *reinterpret_cast<uint4*>(bslot + d1[k]) = lo_first ? lo : hi;
          *reinterpret_cast<uint4*>(bslot + d2[k]) = lo_first ? hi : lo;
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&sm->full_a[slot]);
        if ((s % SPC) == SPC - 1) mbar_arrive(&sm->chunk_free[b]);
      }
      if ((s % SPC) == SPC - 1) bf.next(nbuf);
    }
  } else {
    // ---- producers: two threads per product row ----
    const int t = warp / PWT, h = (warp >> 2) % PPR, q = warp & 3;
    const int lrow = t * 128 + q * 32 + lane;         // row within the CTA's group
    const int mrow = blockIdx.y * NTR + lrow;
    int su = -1, sv = -1, eu = 0, ru = 0, rv = 0;
    float fuv = 0.f;
    if (mrow < P.nmrow) {
      su = P.rx[mrow];
      sv = P.ry[mrow];
      eu = slot_e[su] + slot_e[sv];
      fuv = exp2f_int(14 - eu);
      ru = rf_rot(P.sfield[su]) + 16 * KPT * h;   // rotated cell of this thread's first cell, before the stage offset
      rv = rf_rot(P.sfield[sv]) + 16 * KPT * h;
    }
    if (h == 0) row_e[lrow] = eu;
    const uint32_t lane_addr = tbase + ((uint32_t)(q * 32) << 16);
    Ring st, bf;   // stage slot; chunk buffer (advanced after the chunk's last stage)
    for (int s = 0; s < nst; ++s, st.next(NSA)) {
      const int slot = st.slot;
      const int o = (s % SPC) * AST;
      const int b = bf.slot;
      if ((s % SPC) == 0 && !warp_wait(&sm->full_tma[b], bf.par, limit, abort, status)) break;
      if (s >= NSA && !warp_wait(&sm->empty_a[slot], st.par ^ 1u, limit, abort, status)) break;
      tc_fence_after();
      const float* stage = buf + (size_t)b * P.nstage * SROW;
#pragma unroll
      for (int kk = 0; kk < KPT; ++kk) {
        uint32_t v[16];   // words 0..7: hi of cells 2k, 2k + 1; words 8..15: lo
        if (su >= 0) {
          const float* pa = stage + (size_t)su * SROW;
          const float* pb = stage + (size_t)sv * SROW;
          float4 x[4], y[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            x[u] = *reinterpret_cast<const float4*>(pa + ((o + ru + 16 * kk + 4 * u) & (CHUNK - 1)));
            y[u] = *reinterpret_cast<const float4*>(pb + ((o + rv + 16 * kk + 4 * u) & (CHUNK - 1)));
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            split_f16x2(x[u].x * y[u].x * fuv, x[u].y * y[u].y * fuv, v[2 * u], v[8 + 2 * u]);
            split_f16x2(x[u].z * y[u].z * fuv, x[u].w * y[u].w * fuv, v[2 * u + 1], v[8 + 2 * u + 1]);
          }
        } else {
#pragma unroll
          for (int u = 0; u < 16; ++u) v[u] = 0u;
        }
        tmem_st16(lane_addr + (uint32_t)a_col(N, NT, slot, t, KPT * h + kk), v);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&sm->full_a[slot]);
        if ((s % SPC) == SPC - 1) mbar_arrive(&sm->chunk_free[b]);
      }
      if ((s % SPC) == SPC - 1) bf.next(nbuf);
      if ((s % FLUSH) == FLUSH - 1 || s == nst - 1) {
        if (!warp_wait(&sm->empty_a[slot], st.par, limit, abort, status)) break;
        tc_fence_after();
        // this thread's share of the row's accumulators: columns [h N / PPR, (h + 1) N / PPR), pairs (hi, lo)
        for (int c8 = h * (N / PPR); c8 < (h + 1) * (N / PPR); c8 += 8) {
          uint32_t d[8];
          tmem_ld8_wait(lane_addr + (uint32_t)(t * N + c8), d);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int w = (c8 >> 1) + k;
            if (su >= 0 && w < P.nmcol) {
              const size_t i = (size_t)w * NTR + lrow;
              kahan_add(sums[i], comp[i], __uint_as_float(d[2 * k]) + __uint_as_float(d[2 * k + 1]));
            }
          }
        }
        tc_fence_before();
      }
    }
  }
  __syncthreads();
  if (warp == mw) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(NCOLS) : "memory");
  }
  if (!*abort) {
    // this CTA's sums of every output whose product row lies in this group, unscaled in float64
    double* dst = part + (size_t)blockIdx.x * P.nout;
    for (int oi = tid; oi < P.nout; oi += blockDim.x) {
      const int g = P.gidx[oi];
      if (g < 0) {
        if (blockIdx.y == 0) dst[oi] = 0.0;
        continue;
      }
      const int r = g / P.nmcol, w = g - r * P.nmcol;
      if (r / NTR == (int)blockIdx.y) {
        const int lr = r - (int)blockIdx.y * NTR;
        const size_t i = (size_t)w * NTR + lr;
        dst[oi] = ((double)sums[i] + (double)comp[i]) * exp2d_int(row_e[lr] + col_e[w] - 28);
      }
    }
  }
}
