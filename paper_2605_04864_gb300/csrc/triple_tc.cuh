// Triple products over cells on the 5th-generation tensor cores (tcgen05, TMEM accumulators).
//
// The contraction of Eq. bi_sco / Eq. new_bispec in real space,
//     D[row, col] = sum_x A_i(x) B_j(x) C_col(x)      (row = pair (i, j) of a family, col = k or G),
// is a GEMM with M = rows, N = columns (<= 32) and K = cells.  Per CTA:
//   * NT row tiles of 128 rows (two threads per row, eight warps per tile), one control warp;
//   * the staged fields of a chunk of 128 cells arrive by bulk asynchronous copies (the TMA unit,
//     one 512-byte copy per field) into a ring of two or three shared-memory buffers, completed on an
//     mbarrier with a transaction count;
//   * each producer thread forms its row's pair products P = A_i B_j for 16 of the 32 cells of an A stage,
//     splits them into tf32 hi + lo and writes both straight into tensor memory (tcgen05.st): the A
//     operand never passes through shared memory;
//   * the producers also write the column operand (hi and lo) into shared memory in the canonical
//     K-major layout without swizzle (8 x 16-byte core matrices);
//   * one thread issues, per 8-cell k step and row tile, the three products hi*hi + hi*lo + lo*hi
//     (tcgen05.mma kind::tf32, M = 128, N = 32, A from tensor memory, B from a shared-memory
//     descriptor) into an FP32 accumulator in tensor memory, and commits each A stage to an
//     mbarrier that frees its buffers;
//   * every FLUSH A stages (4096 cells) the producers read the accumulator back (tcgen05.ld),
//     add it into float64 sums in shared memory, and the next products start a fresh accumulator;
//   * at the end each producer writes its row's float64 sums as the CTA's partials
//     part[cta][row][col], reduced in a fixed order by the same kernels as the other paths.
// Every wait is bounded (clock64 against `limit`); on expiry the kernel records NPC_ERR_TIMEOUT in
// the device status word, the other roles leave their loops, the control thread waits (with a fixed
// bound) for its copies and products in flight, and the allocating warp frees tensor memory.
#pragma once

#include <cstdint>

namespace tc {

constexpr int CHUNK = 128;        // cells per bulk-copy chunk (512 bytes per staged field)
constexpr int SROW = CHUNK + 4;   // floats between staged field rows: 16-byte aligned, and rows
                                  // fall 16 bytes apart modulo 128 (conflict-light 16-byte reads)
// 32-cell stages, two in flight: 16-cell stages with three or four in flight measured 0.91 and
// 0.89 ms against 0.79 ms at 256^3 (the per-stage hand-off costs more than the deeper ring saves)
constexpr int AST = 32;           // cells per A stage (k steps of 8)
constexpr int NSA = 2;            // A stages in flight (tensor-memory ring)
constexpr int KSTEPS = AST / 8;
constexpr int SPC = CHUNK / AST;  // A stages per chunk
constexpr int CPT = AST / 2;      // cells per producer thread per A stage (two threads per row)
constexpr int FLUSH = 4096 / AST; // A stages between float64 flushes (4096 cells)
constexpr int NCOL = 32;          // MMA N (columns, padded)
constexpr int BTILE = 1024;       // bytes of one k step of the column operand (32 x 8 tf32)
constexpr long long DRAIN_LIMIT = 1ll << 31;  // cycles a clean-up wait may take

// column of tensor memory holding A stage `sb` (0/1), row tile `t`, part hl (0 hi, 1 lo)
__device__ __forceinline__ uint32_t col_a(int sb, int t, int hl, int nt) { return (uint32_t)(((sb * nt + t) * 2 + hl) * AST); }
__device__ __forceinline__ uint32_t col_d(int t, int nt) { return (uint32_t)(NSA * nt * 2 * AST + t * NCOL); }

__host__ __device__ constexpr uint32_t tmem_cols(int nt) {
  return (nt * (2 * NSA * AST + NCOL)) <= 256 ? 256u : 512u;
}

// instruction descriptor: D f32, A and B tf32, both K-major, N = 32, M = 128
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NCOL >> 3) << 17) | ((128u >> 4) << 24);

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
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of parity `parity`.  Gives up (false) when another role has aborted
// or after `limit` cycles, in which case it records the timeout and raises the CTA's abort flag.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit, volatile int* abort,
                                          int* status) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > limit) {
      *abort = 1;
      atomicCAS(status, 0, (int)NPC_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
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
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]));
}

// 16 columns of this warp's 32 lanes, with the wait in the same statement so that no use of the
// registers can be scheduled before the data has arrived
__device__ __forceinline__ void tmem_ld16_wait(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
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

__device__ __forceinline__ void mma_tf32(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(
          d),
      "r"(a), "l"(bdesc), "r"(IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// hi = v with the 13 low mantissa bits cleared (what the tensor core reads of a tf32 operand),
// lo = v - hi exactly; the product keeps about 21 bits (hi*hi + hi*lo + lo*hi)
__device__ __forceinline__ void split(float v, uint32_t& hi, uint32_t& lo) {
  hi = __float_as_uint(v) & 0xffffe000u;
  lo = __float_as_uint(v - __uint_as_float(hi));
}

struct Smem {
  uint64_t full_tma[3];     // chunk buffer filled (transaction count)
  uint64_t full_a[NSA];     // A stage written by every producer warp
  uint64_t empty_a[NSA];    // products of an A stage complete (tcgen05.commit)
  uint64_t drain;           // clean-up commit
  uint32_t tmem_base;
  int abort;
};

}  // namespace tc

// grid = (CTAs over the cells, row groups of NT x 128 rows); block = NT x 256 producers (two per
// row: warp 8t + 4h + q serves tile t, lanes 32q.. of tensor memory, cells 16h.. of each A stage)
// + one control warp.  Requires ncell % 128 == 0, ncol <= 32; nbuf = 2 or 3 chunk buffers;
// dynamic shared memory = tc_triple_smem(nstage, nbuf, NT).
template <int NT>
__global__ void __launch_bounds__(NT * 256 + 32, 1)
k_triple_tc(const float* __restrict__ R, const __grid_constant__ TripleArgs A, const int* __restrict__ pair_ij,
            const int* __restrict__ row_pair, double* __restrict__ part, int* status, long long limit, int nbuf) {
  using namespace tc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* buf = reinterpret_cast<float*>(smem_raw);                                   // [nbuf][nstage][SROW]
  const size_t buf_bytes = (size_t)nbuf * A.nstage * SROW * sizeof(float);
  unsigned char* btile = smem_raw + ((buf_bytes + 1023) & ~(size_t)1023);     // [NSA sb][2 hl][KSTEPS k][1 KB]
  double* accs = reinterpret_cast<double*>(btile + NSA * 2 * KSTEPS * BTILE);  // [NCOL][NT * 128]
  Smem* sm = reinterpret_cast<Smem*>(accs + (size_t)NCOL * NT * 128);
  volatile int* abort = &sm->abort;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ctrl = NT * 8;  // control warp index
  constexpr uint32_t NCOLS = tmem_cols(NT);

  // cell range of this CTA, in whole chunks
  const int64_t nchunk_all = A.ncell / CHUNK;
  const int64_t per = (nchunk_all + gridDim.x - 1) / gridDim.x;
  const int64_t c_beg = min((int64_t)blockIdx.x * per, nchunk_all);
  const int64_t c_end = min(c_beg + per, nchunk_all);
  const int nchunk = (int)(c_end - c_beg);
  const int nst = nchunk * SPC;
  const int64_t cell0 = c_beg * CHUNK;

  for (int i = tid; i < NCOL * NT * 128; i += blockDim.x) accs[i] = 0.0;
  if (warp == ctrl) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm->tmem_base)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    if (lane == 0) {
      for (int b = 0; b < nbuf; ++b) mbar_init(&sm->full_tma[b], 1);
      for (int b = 0; b < NSA; ++b) {
        mbar_init(&sm->full_a[b], NT * 8);
        mbar_init(&sm->empty_a[b], 1);
      }
      mbar_init(&sm->drain, 1);
      sm->abort = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = sm->tmem_base;

  if (warp == ctrl) {
    if (lane == 0) {
      // ---- control thread: bulk copies of the staged fields, and the tensor-core products ----
      int issued = 0;
      auto issue = [&](int c) {
        const int b = c % nbuf;
        mbar_arrive_tx(&sm->full_tma[b], (uint32_t)(A.nstage * CHUNK * sizeof(float)));
        for (int s = 0; s < A.nstage; ++s)
          bulk_g2s(buf + ((size_t)b * A.nstage + s) * SROW,
                   R + (size_t)A.stage_field[s] * A.ncell + cell0 + (int64_t)c * CHUNK, CHUNK * sizeof(float),
                   &sm->full_tma[b]);
      };
      for (; issued < min(nbuf, nchunk); ++issued) issue(issued);
      const uint64_t bdesc0 = sdesc(smem_u32(btile), 128, 256);
      bool ok = true;
      for (int s = 0; s < nst; ++s) {
        const int sb = s % NSA;
        if (!mbar_wait(&sm->full_a[sb], (uint32_t)((s / NSA) & 1), limit, abort, status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const bool fresh = (s % FLUSH) == 0;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const uint32_t d = tbase + col_d(t, NT);
#pragma unroll
          for (int j = 0; j < KSTEPS; ++j) {
            const uint32_t ahi = tbase + col_a(sb, t, 0, NT) + 8 * j;
            const uint32_t alo = tbase + col_a(sb, t, 1, NT) + 8 * j;
            // the descriptor's start address field counts 16-byte units
            const uint64_t bh = bdesc0 + (uint64_t)((((sb * 2 + 0) * KSTEPS + j) * BTILE) >> 4);
            const uint64_t bl = bdesc0 + (uint64_t)((((sb * 2 + 1) * KSTEPS + j) * BTILE) >> 4);
            mma_tf32(d, ahi, bh, (fresh && j == 0) ? 0u : 1u);
            mma_tf32(d, ahi, bl, 1u);
            mma_tf32(d, alo, bh, 1u);
          }
        }
        mma_commit(&sm->empty_a[sb]);
        // the last A stage of chunk c has been read by every producer: its buffer is free
        if ((s % SPC) == SPC - 1 && issued < nchunk) issue(issued++);
      }
      // every product issued must finish before tensor memory is freed (the producers have waited
      // for them unless a wait gave up)
      mma_commit(&sm->drain);
      mbar_drain(&sm->drain, 0);
      if (!ok || *abort)
        for (int c = max(0, issued - nbuf); c < issued; ++c) mbar_drain(&sm->full_tma[c % nbuf], (uint32_t)((c / nbuf) & 1));
    }
    __syncwarp();
  } else {
    // ---- producers: two threads per row ----
    const int t = warp >> 3, h = (warp >> 2) & 1, q = warp & 3;
    const int lrow = t * 128 + q * 32 + lane;         // row within the CTA's group
    const int row = blockIdx.y * (NT * 128) + lrow;
    int sa = -1, sbs = -1;
    if (row < A.nrows) {
      const int fam = row / A.npair, p = row_pair[row % A.npair];
      const int pij = pair_ij[p];
      sa = A.a_slot[fam][pij & 0xffff];
      sbs = A.b_slot[fam][pij >> 16];
    }
    // the column operand: this warp writes the core matrices cm = warp, warp + 8 NT (< 32);
    // cm % 4 = warp % 4 is the 8-column group, lane / 4 the column within it, lane % 4 the cell
    const int ncol_here = q * 8 + (lane >> 2);
    const int cslot = ncol_here < A.ncol ? A.c_slot[ncol_here] : -1;
    const uint32_t lane_addr = tbase + ((uint32_t)(q * 32) << 16);
    for (int s = 0; s < nst; ++s) {
      const int sb = s % NSA;
      const int c = s / SPC;
      const int o = (s % SPC) * AST;
      const int b = c % nbuf;
      if ((s % SPC) == 0 && !mbar_wait(&sm->full_tma[b], (uint32_t)((c / nbuf) & 1), limit, abort, status))
        break;
      if (s >= NSA && !mbar_wait(&sm->empty_a[sb], (uint32_t)(((s - NSA) / NSA) & 1), limit, abort, status)) break;
      tc_fence_after();
      const float* stage = buf + (size_t)b * A.nstage * SROW;
      // A operand: pair products of this row for cells o + CPT h .. + CPT, hi and lo
      {
        uint32_t vh[CPT], vl[CPT];
        if (sa >= 0) {
          const float4* pa = reinterpret_cast<const float4*>(stage + (size_t)sa * SROW + o + CPT * h);
          const float4* pb = reinterpret_cast<const float4*>(stage + (size_t)sbs * SROW + o + CPT * h);
          float4 x[CPT / 4], y[CPT / 4];
#pragma unroll
          for (int u = 0; u < CPT / 4; ++u) {
            x[u] = pa[u];
            y[u] = pb[u];
          }
#pragma unroll
          for (int u = 0; u < CPT / 4; ++u) {
            split(x[u].x * y[u].x, vh[4 * u + 0], vl[4 * u + 0]);
            split(x[u].y * y[u].y, vh[4 * u + 1], vl[4 * u + 1]);
            split(x[u].z * y[u].z, vh[4 * u + 2], vl[4 * u + 2]);
            split(x[u].w * y[u].w, vh[4 * u + 3], vl[4 * u + 3]);
          }
        } else {
#pragma unroll
          for (int u = 0; u < CPT; ++u) vh[u] = vl[u] = 0u;
        }
        if constexpr (CPT == 16) {
          tmem_st16(lane_addr + col_a(sb, t, 0, NT) + CPT * h, vh);
          tmem_st16(lane_addr + col_a(sb, t, 1, NT) + CPT * h, vl);
        } else {
          tmem_st8(lane_addr + col_a(sb, t, 0, NT) + CPT * h, vh);
          tmem_st8(lane_addr + col_a(sb, t, 1, NT) + CPT * h, vl);
        }
      }
      // B operand: core matrices of 8 columns x 4 cells, k step j = cm / 8, K half kh = (cm / 4) % 2
      for (int cm = warp; cm < 8 * KSTEPS; cm += NT * 8) {
        const int j = cm >> 3, kh = (cm >> 2) & 1;
        const int cell = o + 8 * j + 4 * kh + (lane & 3);
        const float v = cslot >= 0 ? stage[(size_t)cslot * SROW + cell] : 0.f;
        uint32_t hi, lo;
        split(v, hi, lo);
        const size_t off = (size_t)q * 256 + kh * 128 + (lane >> 2) * 16 + (lane & 3) * 4;
        *reinterpret_cast<uint32_t*>(btile + ((sb * 2 + 0) * KSTEPS + j) * BTILE + off) = hi;
        *reinterpret_cast<uint32_t*>(btile + ((sb * 2 + 1) * KSTEPS + j) * BTILE + off) = lo;
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      fence_async_smem();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm->full_a[sb]);
      if ((s % FLUSH) == FLUSH - 1 || s == nst - 1) {
        if (!mbar_wait(&sm->empty_a[sb], (uint32_t)((s / NSA) & 1), limit, abort, status)) break;
        tc_fence_after();
        uint32_t v[16];
        tmem_ld16_wait(lane_addr + col_d(t, NT) + 16 * h, v);
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) accs[(size_t)(16 * h + cc) * (NT * 128) + lrow] += (double)__uint_as_float(v[cc]);
        tc_fence_before();
      }
    }
  }
  __syncthreads();
  if (warp == ctrl) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(NCOLS) : "memory");
  } else if (!*abort) {
    // this CTA's float64 sums as part[cta][row][col]
    const int t = warp >> 3, h = (warp >> 2) & 1, q = warp & 3;
    const int lrow = t * 128 + q * 32 + lane;
    const int row = blockIdx.y * (NT * 128) + lrow;
    if (row < A.nrows) {
      const int fam = row / A.npair, p = row_pair[row % A.npair];
      double* dst = part + ((size_t)blockIdx.x * A.nrows + fam * A.npair + p) * A.ncol;
      for (int cc = 16 * h; cc < 16 * h + 16 && cc < A.ncol; ++cc) dst[cc] = accs[(size_t)cc * (NT * 128) + lrow];
    }
  }
}

// dynamic shared memory of k_triple_tc<NT> for `nstage` staged fields and `nbuf` chunk buffers
inline size_t tc_triple_smem(int nstage, int nbuf, int nt) {
  const size_t buf = (size_t)nbuf * nstage * tc::SROW * sizeof(float);
  return ((buf + 1023) & ~(size_t)1023) + tc::NSA * 2 * tc::KSTEPS * tc::BTILE + sizeof(double) * tc::NCOL * nt * 128 +
         sizeof(tc::Smem);
}
