// Register/shared-memory FFT building blocks (Stockham autosort, radix 8 then 4 or 2).
//
// One transform of length N is computed by TPF = N/8 threads; thread t holds the 8 elements
// t + q*TPF (q = 0..7) both before the first stage and after the last stage, so inputs can be
// loaded straight from global memory into registers and outputs stored straight back; only the
// data exchanges between stages go through shared memory.  Stage with current span Ns and radix R:
// butterfly b (b = t + s*TPF, s < 8/R) reads x[b + r*N/R], multiplies input r by w^(r*(b mod Ns))
// with w = exp(DIR*2*pi*i/(Ns*R)), applies the length-R DFT and writes output r to
// (b div Ns)*Ns*R + (b mod Ns) + r*Ns.  DIR = -1 forward (e^{-i k x}), +1 inverse (unscaled).
#pragma once

#include <type_traits>

#include "npc_internal.cuh"

template <typename C, int DIR>
__device__ __forceinline__ C twiddle(const C* __restrict__ tw, int j) {
  C w = tw[j];
  if (DIR > 0) w.y = -w.y;
  return w;
}

template <typename C>
__device__ __forceinline__ void bfly2(C& a, C& b) {
  const C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// length-4 DFT in natural order on (a0, a1, a2, a3)
template <int DIR, typename C>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  const C b0 = cadd(a0, a2), b2 = csub(a0, a2);
  const C b1 = cadd(a1, a3), b3 = cmul_i<DIR>(csub(a1, a3));
  a0 = cadd(b0, b1);
  a2 = csub(b0, b1);
  a1 = cadd(b2, b3);
  a3 = csub(b2, b3);
}

// length-8 DFT in natural order on v[0..7] (decimation in frequency into two length-4 DFTs)
template <int DIR, typename C>
__device__ __forceinline__ void dft8(C (&v)[8]) {
  using T = decltype(v[0].x);
  const T r = T(0.70710678118654752440);
  C a0 = cadd(v[0], v[4]), a1 = cadd(v[1], v[5]), a2 = cadd(v[2], v[6]), a3 = cadd(v[3], v[7]);
  C c0 = csub(v[0], v[4]);
  C c1 = csub(v[1], v[5]);
  C c2 = csub(v[2], v[6]);
  C c3 = csub(v[3], v[7]);
  // c1 *= w, c2 *= w^2 = DIR*i, c3 *= w^3 with w = exp(DIR*i*pi/4)
  c1 = cmul(c1, cmk(r, T(DIR) * r));
  c2 = cmul_i<DIR>(c2);
  c3 = cmul(c3, cmk(-r, T(DIR) * r));
  dft4<DIR>(a0, a1, a2, a3);
  dft4<DIR>(c0, c1, c2, c3);
  v[0] = a0; v[2] = a1; v[4] = a2; v[6] = a3;
  v[1] = c0; v[3] = c1; v[5] = c2; v[7] = c3;
}

// Shared-memory views used for the inter-stage exchange.  sub(off) is the view of the elements
// from `off` on (off a multiple of 8), used by the sub-transforms of a composite length.
template <typename C> struct ColView {  // element n of column at p[n*stride]
  C* p;
  int stride;
  __device__ __forceinline__ void st(int n, C v) const { p[n * stride] = v; }
  __device__ __forceinline__ C ld(int n) const { return p[n * stride]; }
  __device__ __forceinline__ ColView sub(int off) const { return ColView{p + off * stride, stride}; }
};
template <typename C> struct RowView {  // element n at p[n + n/8] (one pad slot per 8)
  C* p;
  __device__ __forceinline__ static int idx(int n) { return n + (n >> 3); }
  __device__ __forceinline__ void st(int n, C v) const { p[idx(n)] = v; }
  __device__ __forceinline__ C ld(int n) const { return p[idx(n)]; }
  __device__ __forceinline__ RowView sub(int off) const { return RowView{p + idx(off)}; }
};
template <int N> __host__ __device__ constexpr int row_pad_len() { return N + N / 8; }

// Supported transform lengths: powers of two >= 16, and three times a power of two >= 48.
template <int N> struct FftLen {
  static constexpr bool pow2 = (N & (N - 1)) == 0;
  static constexpr int M = pow2 ? N : N / 3;  // power-of-two factor
  static_assert(N >= 16 && (M & (M - 1)) == 0 && (pow2 || (N % 3 == 0 && M >= 16)),
                "transform length must be 2^k >= 16 or 3 * 2^k >= 48");
};

// Rows of length N transformed side by side by THREADS threads, TPF = N/8 per row: G row groups and
// the number of exchange buffers, one per group plus one scratch buffer for the leftover threads
// when TPF does not divide THREADS (they transform zeros so that every thread meets each barrier).
template <int N, int THREADS> struct RowGroups {
  static constexpr int TPF = N / 8;
  static constexpr int G = THREADS / TPF > 0 ? THREADS / TPF : 1;
  static constexpr int NBUF = (THREADS % TPF) ? G + 1 : G;
};

// Barrier among the threads that share one transform's exchange buffer: the whole block (the
// default), one warp (transforms of <= 32 threads packed in a warp), or a named barrier of the
// group's threads (transforms of 64, 128 ... threads) so that row groups do not wait on each other.
struct SyncBlock {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct SyncWarp {
  __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct SyncNamed {
  int id, count;
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
  }
};

// All threads that share `buf` must call this the same number of times (it contains barriers).
// TS: stride into the twiddle table (a length-N/TS sub-transform reads every TS-th twiddle of N).
template <int N, int DIR, int Ns, int TS = 1, typename C, typename View, typename Sync = SyncBlock>
__device__ __forceinline__ void fft_stages(C (&v)[8], const int t, const C* __restrict__ tw,
                                           const View& buf, const Sync& sync = Sync()) {
  constexpr int TPF = N / 8;
  constexpr int REM = N / Ns;
  constexpr int R = (REM >= 8) ? 8 : REM;
  constexpr int BPT = 8 / R;
  static_assert(R == 2 || R == 4 || R == 8, "unsupported radix");
#pragma unroll
  for (int s = 0; s < BPT; ++s) {
    const int b = t + s * TPF;
    if constexpr (Ns > 1) {
      const int k = b & (Ns - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const int j = r * k * (N / (Ns * R));
        v[s + r * BPT] = cmul(v[s + r * BPT], twiddle<C, DIR>(tw, j * TS));
      }
    }
    if constexpr (R == 8) {
      dft8<DIR>(v);
    } else if constexpr (R == 4) {
      dft4<DIR>(v[s], v[s + BPT], v[s + 2 * BPT], v[s + 3 * BPT]);
    } else {
      bfly2(v[s], v[s + BPT]);
    }
  }
  if constexpr (Ns * R < N) {
#pragma unroll
    for (int s = 0; s < BPT; ++s) {
      const int b = t + s * TPF;
      const int base = (b / Ns) * Ns * R + (b & (Ns - 1));
#pragma unroll
      for (int r = 0; r < R; ++r) buf.st(base + r * Ns, v[s + r * BPT]);
    }
    sync();
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = buf.ld(t + q * TPF);
    sync();
    fft_stages<N, DIR, Ns * R, TS>(v, t, tw, buf, sync);
  }
}

// Length-N transform of the elements held in v (thread t of TPF = N/8 threads); `tw` is the
// length-N twiddle table.  For N = 3M (M a power of two) the transform is split by decimation in
// time: the three length-M transforms of x[3m + r] (r = 0, 1, 2) run side by side, one per third
// of the threads, then X[k] = A_0[k mod M] + w^k A_1[k mod M] + w^{2k} A_2[k mod M] with
// w = exp(DIR 2 pi i / N).  Inputs and outputs keep the natural order t + q TPF; the buffer
// holds N elements and may be reused by the caller as soon as this returns.
template <int N, int DIR, typename C, typename View, typename Sync = SyncBlock>
__device__ __forceinline__ void fft_block(C (&v)[8], const int t, const C* __restrict__ tw,
                                          const View& buf, const Sync& sync = Sync()) {
  using L = FftLen<N>;
  if constexpr (L::pow2) {
    fft_stages<N, DIR, 1>(v, t, tw, buf, sync);
  } else {
    constexpr int M = L::M;
    constexpr int TPF = N / 8, SUB = M / 8;
    const int r = t / SUB, s = t % SUB;
#pragma unroll
    for (int q = 0; q < 8; ++q) buf.st(t + q * TPF, v[q]);
    sync();
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = buf.ld(3 * (s + q * SUB) + r);
    sync();
    const View sb = buf.sub(r * M);
    fft_stages<M, DIR, 1, 3>(v, s, tw, sb, sync);
#pragma unroll
    for (int q = 0; q < 8; ++q) sb.st(s + q * SUB, v[q]);
    sync();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = t + q * TPF;
      const int km = k % M;
      const int k2 = (2 * k) % N;
      C a = buf.ld(km);
      a = cadd(a, cmul(buf.ld(M + km), twiddle<C, DIR>(tw, k)));
      a = cadd(a, cmul(buf.ld(2 * M + km), twiddle<C, DIR>(tw, k2)));
      v[q] = a;
    }
    sync();
  }
}

// The barrier a row kernel with THREADS threads uses for its length-N row transforms (TPF = N/8
// threads each, group g): named per group when a group is whole warps, the warp when groups pack
// into warps, else the block.
template <int N, int THREADS> struct RowSync {
  static constexpr int TPF = N / 8;
  static constexpr bool named = (TPF % 32 == 0) && (THREADS % TPF == 0) && (THREADS / TPF <= 15) && (THREADS > TPF);
  static constexpr bool warp = (32 % TPF == 0) && (THREADS % 32 == 0);
  using type = typename std::conditional<named, SyncNamed,
                                         typename std::conditional<warp, SyncWarp, SyncBlock>::type>::type;
  __device__ __forceinline__ static type make(int g) {
    if constexpr (named) return SyncNamed{1 + g, TPF};
    else return type{};
  }
};
