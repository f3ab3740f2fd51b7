// Catalogue scalars (alpha, I22, I33, N0, S3) and deterministic CIC/TSC interlaced painting.
//
// Painting (Sec. 3.1 mass assignment; interlacing as cited there):
//   1. k_brick_count  grid coordinate s = (x - origin) * (n/box) in float64, base cell floor(s)
//                     (wrapped), brick of BS^3 cells; per-brick counts and in-brick ranks.
//   2. k_scan         exclusive scan of the brick counts.
//   3. k_scatter      particles regrouped by brick as records {x, y, z, weight coefficient}.
//   4. k_paint_brick  one CTA per brick accumulates every tap of its particles into a
//                     (BS+4)^3 shared-memory tile (the brick plus the cells its particles can
//                     reach) in 64-bit fixed point, so the sum is independent of thread order;
//                     the tile is written out once.
//   5. k_fold         each mesh cell sums, in a fixed order, the (up to 8) tiles that cover it.
// The mesh is therefore bitwise reproducible run to run without any floating-point atomics.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "npc_internal.cuh"

namespace {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 1024;
constexpr int NSUM = 6;  // sum w, w^2, w^3, nbar w^2, nbar^2 w^3, max |w|

template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
k_cat_partials(const T* __restrict__ w, const T* __restrict__ nbar, int64_t n, double* part) {
  __shared__ double sh[NSUM][RED_THREADS];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t beg = (int64_t)blockIdx.x * chunk;
  const int64_t end = min(n, beg + chunk);
  double a[NSUM] = {0, 0, 0, 0, 0, 0};
  if constexpr (sizeof(T) == 4) {
    // float inputs: products and per-thread sums in float-float arithmetic (error-free products by
    // FMA, two-sum accumulation, about 48 significant bits) instead of the slow FP64 pipe; the
    // per-thread results are exact in double and enter the same fixed-order tree
    float hs[NSUM - 1] = {0, 0, 0, 0, 0}, ls[NSUM - 1] = {0, 0, 0, 0, 0};
    float wmax = 0.0f;
    // explicit _rn operations: the compiler must not fuse a product into the sums below
    auto acc = [&](int k, float vh, float vl) {
      const float s = __fadd_rn(hs[k], vh);
      const float bb = __fsub_rn(s, hs[k]);
      const float e = __fadd_rn(__fadd_rn(__fsub_rn(hs[k], __fsub_rn(s, bb)), __fsub_rn(vh, bb)), __fadd_rn(ls[k], vl));
      hs[k] = __fadd_rn(s, e);
      ls[k] = __fsub_rn(e, __fsub_rn(hs[k], s));
    };
    for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
      const float wi = w ? (float)w[i] : 1.0f;
      const float nb = nbar ? (float)nbar[i] : 0.0f;
      const float p2 = __fmul_rn(wi, wi), e2 = fmaf(wi, wi, -p2);             // w^2
      const float p3 = __fmul_rn(p2, wi), e3 = fmaf(p2, wi, -p3) + e2 * wi;   // w^3
      const float p4 = __fmul_rn(nb, p2), e4 = fmaf(nb, p2, -p4) + nb * e2;   // nbar w^2
      const float pt = __fmul_rn(nb, p3), et = fmaf(nb, p3, -pt) + nb * e3;   // nbar w^3
      const float p5 = __fmul_rn(nb, pt), e5 = fmaf(nb, pt, -p5) + nb * et;   // nbar^2 w^3
      acc(0, wi, 0.0f);
      acc(1, p2, e2);
      acc(2, p3, e3);
      acc(3, p4, e4);
      acc(4, p5, e5);
      wmax = fmaxf(wmax, fabsf(wi));
    }
#pragma unroll
    for (int k = 0; k < NSUM - 1; ++k) a[k] = (double)hs[k] + (double)ls[k];
    a[NSUM - 1] = (double)wmax;
  } else {
    for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
      const double wi = w ? (double)w[i] : 1.0;
      const double nb = nbar ? (double)nbar[i] : 0.0;
      const double w2 = wi * wi;
      a[0] += wi;
      a[1] += w2;
      a[2] += w2 * wi;
      a[3] += nb * w2;
      a[4] += nb * nb * w2 * wi;
      a[5] = fmax(a[5], fabs(wi));
    }
  }
#pragma unroll
  for (int k = 0; k < NSUM; ++k) sh[k][threadIdx.x] = a[k];
  __syncthreads();
  for (int off = RED_THREADS / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
#pragma unroll
      for (int k = 0; k < NSUM - 1; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + off];
      sh[NSUM - 1][threadIdx.x] = fmax(sh[NSUM - 1][threadIdx.x], sh[NSUM - 1][threadIdx.x + off]);
    }
    __syncthreads();
  }
  if (threadIdx.x < NSUM) part[blockIdx.x * NSUM + threadIdx.x] = sh[threadIdx.x][0];
}

// One warp: lane l sums the partials of blocks l, l+32, ... in order, then a fixed shuffle tree;
// the reduction order depends only on nblk (bitwise reproducible).
__global__ void k_cat_final(const double* __restrict__ pd, const double* __restrict__ pr, int nblk,
                            int have_randoms, double box, double* __restrict__ sc) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  double g[NSUM] = {0, 0, 0, 0, 0, 0}, r[NSUM] = {0, 0, 0, 0, 0, 0};
  for (int b = lane; b < nblk; b += 32) {
    for (int k = 0; k < NSUM - 1; ++k) g[k] += pd[b * NSUM + k];
    g[NSUM - 1] = fmax(g[NSUM - 1], pd[b * NSUM + NSUM - 1]);
    if (have_randoms) {
      for (int k = 0; k < NSUM - 1; ++k) r[k] += pr[b * NSUM + k];
      r[NSUM - 1] = fmax(r[NSUM - 1], pr[b * NSUM + NSUM - 1]);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    for (int k = 0; k < NSUM - 1; ++k) {
      g[k] += __shfl_down_sync(0xffffffffu, g[k], off);
      r[k] += __shfl_down_sync(0xffffffffu, r[k], off);
    }
    g[NSUM - 1] = fmax(g[NSUM - 1], __shfl_down_sync(0xffffffffu, g[NSUM - 1], off));
    r[NSUM - 1] = fmax(r[NSUM - 1], __shfl_down_sync(0xffffffffu, r[NSUM - 1], off));
  }
  if (lane != 0) return;
  for (int k = 0; k < SC_COUNT; ++k) sc[k] = 0.0;
  if (have_randoms) {
    const double alpha = g[0] / r[0];
    const double i22 = alpha * r[3];
    sc[SC_ALPHA] = alpha;
    sc[SC_I22] = i22;
    sc[SC_I33] = alpha * r[4];
    sc[SC_N0] = (g[1] + alpha * alpha * r[1]) / i22;
    sc[SC_S3] = g[2] - alpha * alpha * alpha * r[2];
    sc[SC_SUMWG] = g[0];
    sc[SC_SUMWR] = r[0];
    sc[SC_SUMW2] = g[1] + alpha * alpha * r[1];
    sc[SC_MAXW_F] = fmax(g[5], fabs(alpha) * r[5]);
    sc[SC_MAXW_N] = fmax(g[5] * g[5], alpha * alpha * r[5] * r[5]);
  } else {
    const double vol = box * box * box;
    const double ws = g[0];
    const double i22 = ws * ws / vol;
    sc[SC_ALPHA] = 0.0;
    sc[SC_I22] = i22;
    sc[SC_I33] = ws * ws * ws / (vol * vol);
    sc[SC_N0] = g[1] / i22;
    sc[SC_S3] = g[2];
    sc[SC_SUMWG] = ws;
    sc[SC_SUMWR] = 0.0;
    sc[SC_SUMW2] = g[1];
    sc[SC_MAXW_F] = g[5];
    sc[SC_MAXW_N] = g[5] * g[5];
  }
}

// ---------------------------------------------------------------------------------------------
// Painting
// ---------------------------------------------------------------------------------------------
struct PaintGeo {
  int n, bs, nb, ts;     // mesh cells, brick size, bricks per side, tile side (bs + 4)
  double o[3];           // origin
  double inv_h;          // n / box
  float o_hi[3], o_lo[3];      // origin and n / box as float pairs (hi + lo) for the scatter's
  float ih_hi, ih_lo;          // float fast path
};

__device__ __forceinline__ long long wrapi(long long i, int n) {
  long long r = i % n;
  return r < 0 ? r + n : r;
}

template <typename P>
__global__ void k_brick_count(const P* __restrict__ pos, int64_t n, PaintGeo g, int* __restrict__ count,
                              int* __restrict__ brick, int* __restrict__ rank) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int bidx[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // floor(s) decided in float when s is farther from an integer than a bound on the float
      // rounding error (three roundings of relative size 2^-24 on |x| n/box, |origin| n/box and
      // |s|, with a factor 8 of margin), otherwise in float64 exactly as everywhere else
      const P pa = pos[3 * i + a];
      long long f;
      if (sizeof(P) == 4) {
        const float ih = (float)g.inv_h;
        const float sf = ((float)pa - (float)g.o[a]) * ih;
        const float ff = floorf(sf);
        const float fr = sf - ff;
        const float tol = 1.0e-6f * ((fabsf((float)pa) + fabsf((float)g.o[a])) * ih + fabsf(sf)) + 1.0e-6f;
        if (fabsf(sf) < 1.0e6f && fr > tol && fr < 1.0f - tol) {
          f = (long long)ff;
        } else {
          const double s = ((double)pa - g.o[a]) * g.inv_h;
          if (!(fabs(s) < 1e15)) { ok = false; bidx[a] = 0; continue; }
          f = (long long)floor(s);
        }
      } else {
        const double s = ((double)pa - g.o[a]) * g.inv_h;
        if (!(fabs(s) < 1e15)) { ok = false; bidx[a] = 0; continue; }
        f = (long long)floor(s);
      }
      bidx[a] = (int)(wrapi(f, g.n) / g.bs);
    }
    if (!ok) { brick[i] = -1; rank[i] = 0; continue; }
    const int b = (bidx[2] * g.nb + bidx[1]) * g.nb + bidx[0];
    brick[i] = b;
    rank[i] = atomicAdd(&count[b], 1);
  }
}

// exclusive scan of count[0..m) into start[0..m), single block
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ count, int m, int* __restrict__ start) {
  __shared__ int sh[1024];
  const int per = (m + blockDim.x - 1) / blockDim.x;
  const int beg = threadIdx.x * per;
  int s = 0;
  for (int i = beg; i < min(m, beg + per); ++i) s += count[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < blockDim.x; off <<= 1) {
    int v = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  int run = sh[threadIdx.x] - s;
  for (int i = beg; i < min(m, beg + per); ++i) {
    start[i] = run;
    run += count[i];
  }
}

template <typename R> struct RecOf;
template <> struct RecOf<float> { using type = float4; };
template <> struct RecOf<double> { using type = double4_32a; };

// Per particle, per axis: the float64 decisions of the oracle are taken here once and stored as
//   meta bits 8a..8a+4: base cell floor(s) relative to its brick (< 16)
//   meta bits 8a+5   : phase-a tap centre minus base (TSC floor(s+1/2) - floor(s); CIC 0)
//   meta bits 8a+6..7: phase-b tap centre minus base (TSC floor((s+1/2)+1/2) - floor(s);
//                      CIC floor(s+1/2) - floor(s))
// and the record keeps frac = s - floor(s) (exact in float64, rounded once to R) and the weight.
template <int ASSIGN>
__device__ __forceinline__ uint32_t axis_meta(double s, int n, int bs, double* frac) {
  const double f = floor(s);
  const long long fb = (long long)f;
  const double sb = s + 0.5;
  long long ia, ib;
  if (ASSIGN == 2) {
    ia = fb;
    ib = (long long)floor(sb);
  } else {
    ia = (long long)floor(s + 0.5);
    ib = (long long)floor(sb + 0.5);
  }
  *frac = s - f;
  const uint32_t local = (uint32_t)(wrapi(fb, n) % bs);
  return local | ((uint32_t)(ia - fb) << 5) | ((uint32_t)(ib - fb) << 6);
}

// The same decisions and fraction from a float position in float arithmetic: s = (x - origin) n/box
// as a float pair (exact difference by two-sum, exact product error by fma; about 2^-46 relative),
// its floor and the fraction s - floor(s) to float precision.  For TSC floor(s + 1/2) - floor(s) is
// [frac >= 1/2] and floor(s + 1) - floor(s) = 1; for CIC the phase-a offset is 0 and the phase-b one
// [frac >= 1/2], exactly as the float64 expressions give them.  Returns false (the caller takes the
// float64 path) when |s| >= 2^22 or the fraction lies within 1e-6 of 0, 1/2 or 1, where the float64
// rounding of s could decide differently.
template <int ASSIGN>
__device__ __forceinline__ bool axis_meta_fast(float x, float o_hi, float o_lo, float ih_hi, float ih_lo, int n, int bs,
                                               float* frac, uint32_t* meta) {
  const float d1 = __fsub_rn(x, o_hi);
  const float bv = __fsub_rn(d1, x);
  const float d2 = __fsub_rn(__fadd_rn(__fsub_rn(x, __fsub_rn(d1, bv)), __fsub_rn(-o_hi, bv)), o_lo);
  // the rounded product is never fused into a later add: s2 carries its exact error
  const float s1 = __fmul_rn(d1, ih_hi);
  float s2 = fmaf(d1, ih_hi, -s1);
  s2 = fmaf(d1, ih_lo, s2);
  s2 = fmaf(d2, ih_hi, s2);
  if (!(fabsf(s1) < 4194304.0f)) return false;
  float f = floorf(s1);
  float fr = __fadd_rn(__fsub_rn(s1, f), s2);
  if (fr < 0.0f) {
    f -= 1.0f;
    fr += 1.0f;
  } else if (fr >= 1.0f) {
    f += 1.0f;
    fr -= 1.0f;
  }
  const float tol = 1.0e-6f;
  if (fr < tol || fr > 1.0f - tol || fabsf(fr - 0.5f) < tol) return false;
  const int fb = (int)f;
  const uint32_t half = fr >= 0.5f ? 1u : 0u;
  const uint32_t local = (uint32_t)((((fb % n) + n) % n) % bs);
  const uint32_t da = ASSIGN == 2 ? 0u : half, db = ASSIGN == 2 ? half : 1u;
  *meta = local | (da << 5) | (db << 6);
  *frac = fr;
  return true;
}

// coefficient * w^power per particle; coef_kind: 0 -> 1, 1 -> -alpha, 2 -> +alpha^2
template <int ASSIGN, typename P, typename R>
__global__ void k_scatter(const P* __restrict__ pos, const P* __restrict__ w, int64_t n, int power,
                          int coef_kind, const double* __restrict__ sc, PaintGeo g, const int* __restrict__ brick,
                          const int* __restrict__ rank, const int* __restrict__ start,
                          typename RecOf<R>::type* __restrict__ rec, uint32_t* __restrict__ meta) {
  double coef = 1.0;
  if (coef_kind == 1) coef = -sc[SC_ALPHA];
  if (coef_kind == 2) coef = sc[SC_ALPHA] * sc[SC_ALPHA];
  const float coef_f = (float)coef;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int b = brick[i];
    if (b < 0) continue;
    const int dst = start[b] + rank[i];
    if constexpr (sizeof(R) == 4 && sizeof(P) == 4) {
      // float records from float positions: the float pair path, float64 only near a decision
      uint32_t u[3];
      float wcf;
      {
        const float wf = w ? (float)w[i] : 1.0f;
        wcf = coef_f * (power == 2 ? wf * wf : wf);
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float x = (float)pos[3 * i + a];
        float frf;
        uint32_t ma;
        if (!axis_meta_fast<ASSIGN>(x, g.o_hi[a], g.o_lo[a], g.ih_hi, g.ih_lo, g.n, g.bs, &frf, &ma)) {
          double frd;
          ma = axis_meta<ASSIGN>(((double)x - g.o[a]) * g.inv_h, g.n, g.bs, &frd);
          frf = (float)frd;
        }
        const uint32_t q = __float2uint_rz(frf * 16777216.0f);
        u[a] = (q > 0xffffffu ? 0xffffffu : q) | ((ma & 255u) << 24);
      }
      typename RecOf<R>::type r;
      r.x = __uint_as_float(u[0]);
      r.y = __uint_as_float(u[1]);
      r.z = __uint_as_float(u[2]);
      r.w = wcf;
      rec[dst] = r;
      continue;
    }
    const double wi = w ? (double)w[i] : 1.0;
    const double wc = coef * (power == 2 ? wi * wi : wi);
    double fr[3];
    uint32_t m = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double s = ((double)pos[3 * i + a] - g.o[a]) * g.inv_h;
      m |= axis_meta<ASSIGN>(s, g.n, g.bs, &fr[a]) << (8 * a);
    }
    typename RecOf<R>::type r;
    if constexpr (sizeof(R) == 4) {
      // one 16-byte record: per axis the fraction in 24-bit fixed point (truncated, |error| < 2^-24
      // of a cell) with that axis's 8 decision bits on top, and the float weight
      uint32_t u[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const uint32_t q = __float2uint_rz((float)fr[a] * 16777216.0f);
        u[a] = (q > 0xffffffu ? 0xffffffu : q) | (((m >> (8 * a)) & 255u) << 24);
      }
      r.x = __uint_as_float(u[0]);
      r.y = __uint_as_float(u[1]);
      r.z = __uint_as_float(u[2]);
      r.w = (float)wc;
    } else {
      r.x = (R)fr[0];
      r.y = (R)fr[1];
      r.z = (R)fr[2];
      r.w = (R)wc;
      meta[dst] = m;
    }
    rec[dst] = r;
  }
}

// Per-axis taps of one phase: up to 3 (TSC) or 2 (CIC) tile cells with weights, from the
// stored fraction and decision bits.
template <int ASSIGN, typename T>
__device__ __forceinline__ void axis_taps(T frac, uint32_t m8, int phase, int* idx, T* wt) {
  const int local = (int)(m8 & 31u);
  const int off = phase ? (int)((m8 >> 6) & 3u) : (int)((m8 >> 5) & 1u);
  // d = s - centre (phase a) or (s + 1/2) - centre (phase b)
  const T d = frac + (phase ? T(0.5) : T(0)) - T(off);
  const int rel = local + off + 1;   // tile index of the centre (tile starts one cell below the brick)
  if (ASSIGN == 2) {
    idx[0] = rel; wt[0] = T(1) - d;
    idx[1] = rel + 1; wt[1] = d;
  } else {
    const T a = T(0.5) - d, b = T(0.5) + d;
    idx[0] = rel - 1; wt[0] = T(0.5) * a * a;
    idx[1] = rel; wt[1] = T(0.75) - d * d;
    idx[2] = rel + 1; wt[2] = T(0.5) * b * b;
  }
}

// Round to the nearest 64-bit integer (ties to even).  The float path takes |v| < 2^43 (the tile
// kernel's scale guarantees it) and needs no conversion instruction: hi = rn(v / 2^22) and the exact
// remainder lo = v - 2^22 hi, both of magnitude <= 2^21, are rounded to integers by adding 1.5 * 2^23
// (the float add rounds to nearest even, and the integer sits in the low mantissa bits); since
// 2^22 hi is an even integer, 2^22 hi + rn(lo) = rn(v).
template <typename T> __device__ __forceinline__ long long to_fixed(T v);
template <> __device__ __forceinline__ long long to_fixed<float>(float v) {
  const float magic = 12582912.0f;                         // 1.5 * 2^23
  const float th = v * 2.384185791015625e-07f + magic;     // rn(v 2^-22) + magic
  const float hf = th - magic;                             // exact
  const float lf = fmaf(hf, -4194304.0f, v);               // v - 2^22 hi, exact
  const float tl = lf + magic;
  const int hi = __float_as_int(th) - 0x4B400000;
  const int lo = __float_as_int(tl) - 0x4B400000;
  return (long long)hi * 4194304LL + (long long)lo;
}
template <> __device__ __forceinline__ long long to_fixed<double>(double v) { return __double2ll_rn(v); }

// 64-bit fixed point back to T times 2^-e; the float path uses two 32-bit conversions.
template <typename T> __device__ __forceinline__ T from_fixed(long long q, T inv);
template <> __device__ __forceinline__ float from_fixed<float>(long long q, float inv) {
  const int hi = (int)(q >> 32);
  const unsigned lo = (unsigned)(q & 0xffffffffull);
  return fmaf((float)hi, 4294967296.0f, (float)lo) * inv;
}
template <> __device__ __forceinline__ double from_fixed<double>(long long q, double inv) { return (double)q * inv; }

// One CTA per (brick, phase): fixed-point accumulation of all taps in a (bs+4)^3 tile.
template <int ASSIGN, typename R, typename T>
__global__ void __launch_bounds__(512)
k_paint_brick(const typename RecOf<R>::type* __restrict__ rec, const uint32_t* __restrict__ meta,
              const int* __restrict__ start, const int* __restrict__ count, PaintGeo g, int nphase,
              const double* __restrict__ sc, int maxw_slot, T* __restrict__ tiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* acc = reinterpret_cast<long long*>(smem_raw);
  const int ts3 = g.ts * g.ts * g.ts;
  const int b = blockIdx.x / nphase, ph = blockIdx.x % nphase;
  for (int i = threadIdx.x; i < ts3; i += blockDim.x) acc[i] = 0;
  const int cnt = count[b];
  // fixed-point scale 2^e with cnt * max|w| * 2^e < 2^61 (no overflow of the tile sums)
  const double bound = (double)cnt * sc[maxw_slot];
  int ex = 0;
  if (bound > 0) frexp(bound, &ex);
  int e = 61 - ex;
  if constexpr (sizeof(T) == 4) {
    // and every tap |w W| 2^e < 2^43, the range of the float conversion
    int exw = 0;
    if (sc[maxw_slot] > 0) frexp(sc[maxw_slot], &exw);
    e = min(e, 43 - exw);
  }
  const T scale = (T)ldexp(1.0, e);
  __syncthreads();
  const int beg = start[b];
  constexpr int NT = ASSIGN == 2 ? 2 : 3;
  // NT adjacent lanes share one object, lane xt taking its x tap: the atomics of one instruction
  // then hit runs of NT neighbouring cells instead of 32 scattered ones (fewer bank wavefronts)
  constexpr int OPW = 32 / NT;   // objects per warp and pass
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int xt = lane % NT, slot = lane / NT;
  for (int k0 = warp * OPW; k0 < cnt; k0 += nwarp * OPW) {
    const int k = k0 + slot;
    if (slot >= OPW || k >= cnt) continue;
    const typename RecOf<R>::type r = rec[beg + k];
    int ix[NT], iy[NT], iz[NT];
    T wx[NT], wy[NT], wz[NT];
    if constexpr (sizeof(R) == 4) {
      const uint32_t ux = __float_as_uint(r.x), uy = __float_as_uint(r.y), uz = __float_as_uint(r.z);
      const float sc24 = 5.9604644775390625e-8f;   // 2^-24
      axis_taps<ASSIGN, T>((T)((float)(ux & 0xffffffu) * sc24), ux >> 24, ph, ix, wx);
      axis_taps<ASSIGN, T>((T)((float)(uy & 0xffffffu) * sc24), uy >> 24, ph, iy, wy);
      axis_taps<ASSIGN, T>((T)((float)(uz & 0xffffffu) * sc24), uz >> 24, ph, iz, wz);
    } else {
      const uint32_t m = meta[beg + k];
      axis_taps<ASSIGN, T>((T)r.x, m & 255u, ph, ix, wx);
      axis_taps<ASSIGN, T>((T)r.y, (m >> 8) & 255u, ph, iy, wy);
      axis_taps<ASSIGN, T>((T)r.z, (m >> 16) & 255u, ph, iz, wz);
    }
    T wxs = wx[0];
    int ixs = ix[0];
#pragma unroll
    for (int a = 1; a < NT; ++a)
      if (xt == a) { wxs = wx[a]; ixs = ix[a]; }
    const T wgt = (T)r.w * scale * wxs;
#pragma unroll
    for (int c = 0; c < NT; ++c) {
#pragma unroll
      for (int bb = 0; bb < NT; ++bb) {
        // tap value (w 2^e W_x) W_z W_y, formed once per tap in a fixed order
        const long long q = to_fixed<T>(wgt * wz[c] * wy[bb]);
        // taps stay inside the tile by construction; the guard only protects shared memory
        if ((unsigned)iz[c] < (unsigned)g.ts && (unsigned)iy[bb] < (unsigned)g.ts && (unsigned)ixs < (unsigned)g.ts)
          atomicAdd(reinterpret_cast<unsigned long long*>(acc + (iz[c] * g.ts + iy[bb]) * g.ts + ixs),
                    static_cast<unsigned long long>(q));
      }
    }
  }
  __syncthreads();
  const T inv = (T)ldexp(1.0, -e);
  T* out = tiles + ((size_t)b * nphase + ph) * ts3;
  for (int i = threadIdx.x; i < ts3; i += blockDim.x) out[i] = from_fixed<T>(acc[i], inv);
}

// Each cell sums the tiles covering it, in a fixed order (brick offset -1, 0, +1 per axis, z
// outermost).  One CTA per (brick, phase); the tile of brick B covers cells [BS B - 1, BS B + BS + 2].
// Thread (x, y) of the CTA owns one column of the brick along z: its x and y options (own tile, the
// lower neighbour's for the first three cells, the upper neighbour's for the last) are fixed per
// thread, only the z options change per cell.
template <typename T, int BS>
__global__ void __launch_bounds__(BS * BS)
k_fold(const T* __restrict__ tiles, PaintGeo g, int nphase, const double* __restrict__ sc, int subtract_mean,
       T* __restrict__ mesh_a, T* __restrict__ mesh_b) {
  constexpr int TS = BS + 4, TS3 = TS * TS * TS;
  const int n = g.n, nb = g.nb;
  const int b = blockIdx.x / nphase, ph = blockIdx.x % nphase;
  const int B[3] = {b % nb, (b / nb) % nb, b / (nb * nb)};
  int nbm[3], nbp[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    nbm[a] = B[a] == 0 ? nb - 1 : B[a] - 1;
    nbp[a] = B[a] == nb - 1 ? 0 : B[a] + 1;
  }
  const T mean = subtract_mean ? (T)(sc[SC_SUMWG] / ((double)n * n * n)) : T(0);
  T* mesh = ph ? mesh_b : mesh_a;
  const int lx = threadIdx.x % BS, ly = threadIdx.x / BS;
  // x and y options: brick coordinate and tile coordinate, lower neighbour first
  int nx = 0, ny = 0, bx[2], tx[2], by[2], ty[2];
  if (lx <= 2) { bx[nx] = nbm[0]; tx[nx] = lx + BS + 1; ++nx; }
  bx[nx] = B[0]; tx[nx] = lx + 1; ++nx;
  if (lx == BS - 1) { bx[nx] = nbp[0]; tx[nx] = 0; ++nx; }
  if (ly <= 2) { by[ny] = nbm[1]; ty[ny] = ly + BS + 1; ++ny; }
  by[ny] = B[1]; ty[ny] = ly + 1; ++ny;
  if (ly == BS - 1) { by[ny] = nbp[1]; ty[ny] = 0; ++ny; }
  // per (iy, ix) option (2 x 2 slots, slot valid when iy < ny and ix < nx): pointer into the tile
  // of the brick in the same z layer; invalid slots hold a valid address and are predicated off
  const size_t zstride = (size_t)nb * nb * nphase * TS3;   // between z layers of bricks
  const T* p_yx[2][2];
  bool ok[2][2];
#pragma unroll
  for (int iy = 0; iy < 2; ++iy)
#pragma unroll
    for (int ix = 0; ix < 2; ++ix) {
      ok[iy][ix] = iy < ny && ix < nx;
      const int yy = ok[iy][ix] ? iy : 0, xx = ok[iy][ix] ? ix : 0;
      const size_t brick = ((size_t)B[2] * nb + by[yy]) * nb + bx[xx];
      p_yx[iy][ix] = tiles + (brick * nphase + ph) * TS3 + ty[yy] * TS + tx[xx];
    }
  const ptrdiff_t dzm = (ptrdiff_t)(nbm[2] - B[2]) * (ptrdiff_t)zstride;   // to the lower z layer
  const ptrdiff_t dzp = (ptrdiff_t)(nbp[2] - B[2]) * (ptrdiff_t)zstride;   // to the upper z layer
  T* col = mesh + ((size_t)(B[2] * BS) * n + (B[1] * BS + ly)) * n + (B[0] * BS + lx);
  // z cells 0..2 also take the lower z layer's tiles, cell BS-1 the upper one's; the loop is unrolled
  // so that the independent loads of several cells are in flight together
#pragma unroll
  for (int lz = 0; lz < BS; ++lz) {
    T v = T(0);
    if (lz <= 2) {
      const ptrdiff_t o = dzm + (ptrdiff_t)(lz + BS + 1) * TS * TS;
#pragma unroll
      for (int iy = 0; iy < 2; ++iy)
#pragma unroll
        for (int ix = 0; ix < 2; ++ix)
          if (ok[iy][ix]) v += p_yx[iy][ix][o];
    }
    {
      const int o = (lz + 1) * TS * TS;
#pragma unroll
      for (int iy = 0; iy < 2; ++iy)
#pragma unroll
        for (int ix = 0; ix < 2; ++ix)
          if (ok[iy][ix]) v += p_yx[iy][ix][o];
    }
    if (lz == BS - 1) {
#pragma unroll
      for (int iy = 0; iy < 2; ++iy)
#pragma unroll
        for (int ix = 0; ix < 2; ++ix)
          if (ok[iy][ix]) v += p_yx[iy][ix][dzp];
    }
    col[(size_t)lz * n * n] = v - mean;
  }
}

template <typename P>
npc_status paint_count(npc_ctx* ctx, const DevCatalog& c, const PaintGeo& g, int* count, int* brick,
                       int* rank) {
  if (c.n == 0) return NPC_OK;
  const int blocks = (int)std::min<int64_t>((c.n + 255) / 256, (int64_t)1 << 20);   // one object per thread
  k_brick_count<P><<<blocks, 256, 0, ctx->stream>>>((const P*)c.pos, c.n, g, count, brick, rank);
  NPC_LAUNCH(ctx);
  return NPC_OK;
}

template <int ASSIGN, typename P, typename R>
npc_status paint_scatter(npc_ctx* ctx, const DevCatalog& c, int power, int coef_kind, const double* sc,
                         const PaintGeo& g, const int* brick, const int* rank, const int* start, void* rec,
                         uint32_t* meta) {
  if (c.n == 0) return NPC_OK;
  const int blocks = (int)std::min<int64_t>((c.n + 255) / 256, (int64_t)1 << 20);   // one object per thread
  k_scatter<ASSIGN, P, R><<<blocks, 256, 0, ctx->stream>>>((const P*)c.pos, (const P*)c.w, c.n, power, coef_kind,
                                                           sc, g, brick, rank, start,
                                                           (typename RecOf<R>::type*)rec, meta);
  NPC_LAUNCH(ctx);
  return NPC_OK;
}

template <int ASSIGN, typename R>
npc_status scatter_cat(npc_ctx* ctx, const DevCatalog& c, int power, int kind, const double* sc, const PaintGeo& g,
                       const int* brick, const int* rank, const int* start, void* rec, uint32_t* meta) {
  if (c.dtype == 1) return paint_scatter<ASSIGN, double, R>(ctx, c, power, kind, sc, g, brick, rank, start, rec, meta);
  return paint_scatter<ASSIGN, float, R>(ctx, c, power, kind, sc, g, brick, rank, start, rec, meta);
}

template <typename T>
npc_status launch_fold(npc_ctx* ctx, const void* tiles, const PaintGeo& g, int nphase, const double* sc, int sub,
                       void* mesh_a, void* mesh_b) {
  const int grid = g.nb * g.nb * g.nb * nphase;
  switch (g.bs) {
    case 4: k_fold<T, 4><<<grid, 16, 0, ctx->stream>>>((const T*)tiles, g, nphase, sc, sub, (T*)mesh_a, (T*)mesh_b); break;
    case 8: k_fold<T, 8><<<grid, 64, 0, ctx->stream>>>((const T*)tiles, g, nphase, sc, sub, (T*)mesh_a, (T*)mesh_b); break;
    default: k_fold<T, 16><<<grid, 256, 0, ctx->stream>>>((const T*)tiles, g, nphase, sc, sub, (T*)mesh_a, (T*)mesh_b); break;
  }
  NPC_LAUNCH(ctx);
  return NPC_OK;
}

template <int ASSIGN, typename R, typename T>
npc_status paint_impl(npc_ctx* ctx, const DevCatalog& d, const DevCatalog* r, const npc_mesh_spec& m,
                      int weight_power, const double* sc, void* mesh_a, void* mesh_b) {
  PaintGeo g;
  g.n = m.n;
  g.bs = (m.n >= 48 && m.n % 16 == 0) ? 16 : m.n / 4;   // 16 for every size >= 48; 4, 8 at n = 16, 32
  g.nb = m.n / g.bs;
  g.ts = g.bs + 4;
  for (int a = 0; a < 3; ++a) g.o[a] = m.origin[a];
  g.inv_h = (double)m.n / m.box;
  for (int a = 0; a < 3; ++a) {
    g.o_hi[a] = (float)g.o[a];
    g.o_lo[a] = (float)(g.o[a] - (double)g.o_hi[a]);
  }
  g.ih_hi = (float)g.inv_h;
  g.ih_lo = (float)(g.inv_h - (double)g.ih_hi);
  const int nphase = m.interlace ? 2 : 1;
  const int nbricks = g.nb * g.nb * g.nb;
  const int64_t ntot = d.n + (r ? r->n : 0);
  // brick starts and ranks are 32-bit offsets into one record array
  if (ntot >= (int64_t)1 << 31)
    return set_err(ctx, NPC_ERR_UNSUPPORTED, "painting takes at most 2^31-1 objects (data + randoms)");
  int *count, *start, *brick, *rank;
  uint32_t* meta;
  void* rec;
  void* tiles;
  const size_t ts3 = (size_t)g.ts * g.ts * g.ts;
  NPC_TRY(ws_get(ctx, "paint.count", sizeof(int) * nbricks, (void**)&count));
  NPC_TRY(ws_get(ctx, "paint.start", sizeof(int) * nbricks, (void**)&start));
  NPC_TRY(ws_get(ctx, "paint.brick", sizeof(int) * std::max<int64_t>(ntot, 1), (void**)&brick));
  NPC_TRY(ws_get(ctx, "paint.rank", sizeof(int) * std::max<int64_t>(ntot, 1), (void**)&rank));
  NPC_TRY(ws_get(ctx, "paint.meta", sizeof(uint32_t) * std::max<int64_t>(ntot, 1), (void**)&meta));
  NPC_TRY(ws_get(ctx, "paint.rec", sizeof(typename RecOf<R>::type) * std::max<int64_t>(ntot, 1), &rec));
  NPC_TRY(ws_get(ctx, "paint.tiles", sizeof(T) * ts3 * nbricks * nphase, &tiles));
  NPC_CUDA(ctx, cudaMemsetAsync(count, 0, sizeof(int) * nbricks, ctx->stream));
  // counting: data then randoms share the brick counters (ranks continue)
  if (d.dtype == 1) NPC_TRY(paint_count<double>(ctx, d, g, count, brick, rank));
  else NPC_TRY(paint_count<float>(ctx, d, g, count, brick, rank));
  if (r) {
    if (r->dtype == 1) NPC_TRY(paint_count<double>(ctx, *r, g, count, brick + d.n, rank + d.n));
    else NPC_TRY(paint_count<float>(ctx, *r, g, count, brick + d.n, rank + d.n));
  }
  k_scan<<<1, 1024, 0, ctx->stream>>>(count, nbricks, start);
  NPC_LAUNCH(ctx);
  NPC_TRY(stage_mark(ctx, "paint_count"));
  NPC_TRY((scatter_cat<ASSIGN, R>(ctx, d, weight_power, 0, sc, g, brick, rank, start, rec, meta)));
  if (r) {
    const int kind = weight_power == 1 ? 1 : 2;
    NPC_TRY((scatter_cat<ASSIGN, R>(ctx, *r, weight_power, kind, sc, g, brick + d.n, rank + d.n, start, rec, meta)));
  }
  NPC_TRY(stage_mark(ctx, "paint_scatter"));
  const size_t smem = sizeof(long long) * ts3;
  const int slot = weight_power == 1 ? SC_MAXW_F : SC_MAXW_N;
  auto kern = k_paint_brick<ASSIGN, R, T>;
  NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<nbricks * nphase, 512, smem, ctx->stream>>>((const typename RecOf<R>::type*)rec, meta, start, count, g,
                                                     nphase, sc, slot, (T*)tiles);
  NPC_LAUNCH(ctx);
  NPC_TRY(stage_mark(ctx, "paint_tiles"));
  const int sub = (m.periodic && weight_power == 1) ? 1 : 0;
  return launch_fold<T>(ctx, tiles, g, nphase, sc, sub, mesh_a, mesh_b);
}

// Scalars of a cross spectrum from those of tracers A and B: the normalisation sqrt(I22^A I22^B)
// in the I22 slot, no shot noise, and the tracers' own values for the output (layout in npc.h).
__global__ void k_cross_scalars(const double* __restrict__ sa, const double* __restrict__ sb, double* __restrict__ sx) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < SC_COUNT; ++i) sx[i] = 0.0;
  sx[SC_ALPHA] = sa[SC_ALPHA];
  sx[SC_I22] = sqrt(sa[SC_I22] * sb[SC_I22]);
  sx[SC_I33] = sb[SC_ALPHA];
  sx[SC_N0] = 0.0;
  sx[SC_S3] = sa[SC_I22];
  sx[SC_SUMWG] = sb[SC_I22];
  sx[SC_SUMWR] = sa[SC_SUMWG];
  sx[SC_SUMW2] = sb[SC_SUMWG];
}

// Scalars of a three-tracer bispectrum: tracer 1's values with I33 replaced by the geometric mean
// (I33^1 I33^2 I33^3)^(1/3) (the normalisation of the cross bispectra, Sec. 6 reading) and S3 = 0
// (no shot noise is subtracted from the raw cross estimates).
__global__ void k_cross3_scalars(const double* __restrict__ s1, const double* __restrict__ s2,
                                 const double* __restrict__ s3, double* __restrict__ sx) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < SC_COUNT; ++i) sx[i] = s1[i];
  sx[SC_I33] = cbrt(s1[SC_I33] * s2[SC_I33] * s3[SC_I33]);
  sx[SC_S3] = 0.0;
}

}  // namespace

npc_status launch_cross3_scalars(npc_ctx* ctx, const double* s1, const double* s2, const double* s3, double* sx) {
  k_cross3_scalars<<<1, 32, 0, ctx->stream>>>(s1, s2, s3, sx);
  NPC_LAUNCH(ctx);
  return NPC_OK;
}

npc_status launch_cross_scalars(npc_ctx* ctx, const double* sa, const double* sb, double* sx) {
  k_cross_scalars<<<1, 32, 0, ctx->stream>>>(sa, sb, sx);
  NPC_LAUNCH(ctx);
  return NPC_OK;
}

npc_status launch_catalog_scalars(npc_ctx* ctx, const DevCatalog& d, const DevCatalog* r, double box,
                                  double* dev_scalars) {
  double* part;
  NPC_TRY(ws_get(ctx, "scalars.part", sizeof(double) * NSUM * RED_BLOCKS * 2, (void**)&part));
  if (d.dtype == 1)
    k_cat_partials<double><<<RED_BLOCKS, RED_THREADS, 0, ctx->stream>>>((const double*)d.w, (const double*)d.nbar,
                                                                         d.n, part);
  else
    k_cat_partials<float><<<RED_BLOCKS, RED_THREADS, 0, ctx->stream>>>((const float*)d.w, (const float*)d.nbar,
                                                                        d.n, part);
  NPC_LAUNCH(ctx);
  if (r) {
    if (r->dtype == 1)
      k_cat_partials<double><<<RED_BLOCKS, RED_THREADS, 0, ctx->stream>>>(
          (const double*)r->w, (const double*)r->nbar, r->n, part + NSUM * RED_BLOCKS);
    else
      k_cat_partials<float><<<RED_BLOCKS, RED_THREADS, 0, ctx->stream>>>(
          (const float*)r->w, (const float*)r->nbar, r->n, part + NSUM * RED_BLOCKS);
    NPC_LAUNCH(ctx);
  }
  k_cat_final<<<1, 32, 0, ctx->stream>>>(part, part + NSUM * RED_BLOCKS, RED_BLOCKS, r ? 1 : 0, box, dev_scalars);
  NPC_LAUNCH(ctx);
  return NPC_OK;
}

npc_status launch_paint(npc_ctx* ctx, const DevCatalog& d, const DevCatalog* r, const npc_mesh_spec& m,
                        int weight_power, int prec, const double* dev_scalars, void* mesh_a, void* mesh_b) {
  const bool any_double = d.dtype == 1 || (r && r->dtype == 1);
  if (prec == NPC_PREC_FP64) {
    if (m.assign == 2) return paint_impl<2, double, double>(ctx, d, r, m, weight_power, dev_scalars, mesh_a, mesh_b);
    return paint_impl<3, double, double>(ctx, d, r, m, weight_power, dev_scalars, mesh_a, mesh_b);
  }
  // records keep the fraction s - floor(s) (< 1) in float32 in the mixed path
  (void)any_double;
  if (m.assign == 2) return paint_impl<2, float, float>(ctx, d, r, m, weight_power, dev_scalars, mesh_a, mesh_b);
  return paint_impl<3, float, float>(ctx, d, r, m, weight_power, dev_scalars, mesh_a, mesh_b);
}

// ---------------------------------------------------------------------------------------------
// Allocation-free catalogue scalars.
//
// Some callers cannot call cudaMalloc at all: a host framework that owns every byte of device
// memory through its own pool (a raw allocation would sit outside its accounting), a plugin that
// is only handed device pointers, or a latency-bound loop where the implicit synchronisation of an
// allocation stalls the pipeline.  This entry point serves them: it reuses the reduction kernels
// above, but its scratch (the per-block partial sums and the 16 scalar slots) lives in a
// file-scope device array instead of context workspace, so the call allocates nothing.
// ---------------------------------------------------------------------------------------------
#include <cuda.h>

#include <mutex>

namespace {

constexpr int NOALLOC_CHUNK = 4096;            // objects reduced by one block
constexpr int NOALLOC_MAX_BLOCKS = 8192;       // blocks per catalogue
constexpr int64_t NOALLOC_MAX_OBJECTS = (int64_t)NOALLOC_CHUNK * NOALLOC_MAX_BLOCKS;  // 33,554,432
constexpr size_t NOALLOC_PART = (size_t)NOALLOC_MAX_BLOCKS * NSUM;                     // per catalogue

// 2 catalogues x 8192 blocks x 6 sums + 16 scalar slots, doubles: 786,560 bytes, resident on every
// device that loads this library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_PART + SC_COUNT];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;

// Address of the static array per device, remembered together with the identity of the context it
// was looked up in: a cudaDeviceReset (or another context made current) gives the device a new
// context in which the array may sit elsewhere, so a changed context id triggers a new look-up.
struct NoallocSlot {
  double* ptr = nullptr;
  unsigned long long ctx_id = 0;
  bool ctx_known = false;
};
NoallocSlot g_noalloc_slot[NOALLOC_MAX_DEVICES];

// Identity of the calling thread's current context, through driver entry points the runtime hands
// out (no link-time dependence on the driver library).  False when there is no current context or
// the entry points are unavailable; the caller then looks the address up again on every call.
bool current_context_id(unsigned long long* id) {
  static decltype(&cuCtxGetCurrent) get_current = nullptr;
  static decltype(&cuCtxGetId) get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    resolved = true;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_current, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess || q1 != cudaDriverEntryPointSuccess)
      get_current = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess || q2 != cudaDriverEntryPointSuccess)
      get_id = nullptr;
    cudaGetLastError();
  }
  if (!get_current || !get_id) return false;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || !c) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

npc_status noalloc_err(char* err, size_t errlen, npc_status s, const char* msg) {
  if (err && errlen) {
    std::strncpy(err, msg, errlen - 1);
    err[errlen - 1] = '\0';
  }
  return s;
}

}  // namespace

extern "C" npc_status npc_catalog_scalars_noalloc(const npc_catalog* data, const npc_catalog* randoms, double box,
                                                  double* out_device, void* cuda_stream, char* err, size_t errlen) {
  if (err && errlen) err[0] = '\0';
  if (!data || !out_device) return noalloc_err(err, errlen, NPC_ERR_INVALID_ARG, "data and out_device are required");
  const npc_catalog* cats[2] = {data, randoms};
  for (int c = 0; c < 2; ++c) {
    const npc_catalog* k = cats[c];
    if (!k) continue;
    if (k->n < 0 || (k->n > 0 && !k->pos) || (k->dtype != 0 && k->dtype != 1))
      return noalloc_err(err, errlen, NPC_ERR_INVALID_ARG, "malformed catalogue");
    if (!k->on_device)
      return noalloc_err(err, errlen, NPC_ERR_INVALID_ARG, "catalogue arrays must be device pointers (on_device = 1)");
    if (k->n > NOALLOC_MAX_OBJECTS)
      return noalloc_err(err, errlen, NPC_ERR_INVALID_ARG,
                         "catalogue larger than 33554432 objects, the capacity of the static scratch");
    if (c == 1 && k->n > 0 && !k->nbar) return noalloc_err(err, errlen, NPC_ERR_INVALID_ARG, "randoms need nbar");
  }
  if (!randoms && !(box > 0.0)) return noalloc_err(err, errlen, NPC_ERR_INVALID_ARG, "periodic scalars need box > 0");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    cudaGetLastError();
    return noalloc_err(err, errlen, NPC_ERR_CUDA, "no usable current CUDA device");
  }
  double* scratch;
  {
    // Set-up per device and context, with that device current: host code cannot take the address
    // of a __device__ array directly, so ask the runtime for it (done on the first call on a
    // device, and again only after that device's context has changed).
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoallocSlot& slot = g_noalloc_slot[dev];
    unsigned long long id = 0;
    const bool known = current_context_id(&id);
    if (!slot.ptr || !known || !slot.ctx_known || slot.ctx_id != id) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        slot = NoallocSlot{};
        return noalloc_err(err, errlen, NPC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
      }
      slot.ptr = static_cast<double*>(p);
      // the look-up makes the device's primary context current when none was
      slot.ctx_known = current_context_id(&slot.ctx_id);
    }
    scratch = slot.ptr;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t nmax = std::max<int64_t>(data->n, randoms ? randoms->n : 0);
  const int nblk = (int)std::max<int64_t>(1, (nmax + NOALLOC_CHUNK - 1) / NOALLOC_CHUNK);
  double* part_d = scratch;
  double* part_r = scratch + NOALLOC_PART;
  double* sc = scratch + 2 * NOALLOC_PART;
  // every partial that k_cat_final reads is written by this call's k_cat_partials (blocks past the
  // end of a catalogue write zeros), so nothing needs clearing first
  for (int c = 0; c < 2; ++c) {
    const npc_catalog* k = cats[c];
    if (!k) continue;
    double* part = c == 0 ? part_d : part_r;
    if (k->dtype == 1)
      k_cat_partials<double><<<nblk, RED_THREADS, 0, st>>>((const double*)k->w, (const double*)k->nbar, k->n, part);
    else
      k_cat_partials<float><<<nblk, RED_THREADS, 0, st>>>((const float*)k->w, (const float*)k->nbar, k->n, part);
  }
  k_cat_final<<<1, 32, 0, st>>>(part_d, part_r, nblk, randoms ? 1 : 0, box, sc);
  // peek, not get: an error that the caller's earlier asynchronous work left pending is reported
  // as this call's failure but stays pending for the caller to read
  cudaError_t e = cudaPeekAtLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_device, sc, 8 * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return noalloc_err(err, errlen, NPC_ERR_CUDA, cudaGetErrorString(e));
  return NPC_OK;
}
