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
#include <cmath>

#include "npc_internal.cuh"

namespace {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 256;
constexpr int NSUM = 6;  // sum w, w^2, w^3, nbar w^2, nbar^2 w^3, max |w|

template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
k_cat_partials(const T* __restrict__ w, const T* __restrict__ nbar, int64_t n, double* part) {
  __shared__ double sh[NSUM][RED_THREADS];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t beg = (int64_t)blockIdx.x * chunk;
  const int64_t end = min(n, beg + chunk);
  double a[NSUM] = {0, 0, 0, 0, 0, 0};
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

__global__ void k_cat_final(const double* __restrict__ pd, const double* __restrict__ pr, int nblk,
                            int have_randoms, double box, double* __restrict__ sc) {
  if (threadIdx.x != 0) return;
  double g[NSUM] = {0, 0, 0, 0, 0, 0}, r[NSUM] = {0, 0, 0, 0, 0, 0};
  for (int b = 0; b < nblk; ++b) {
    for (int k = 0; k < NSUM - 1; ++k) g[k] += pd[b * NSUM + k];
    g[NSUM - 1] = fmax(g[NSUM - 1], pd[b * NSUM + NSUM - 1]);
    if (have_randoms) {
      for (int k = 0; k < NSUM - 1; ++k) r[k] += pr[b * NSUM + k];
      r[NSUM - 1] = fmax(r[NSUM - 1], pr[b * NSUM + NSUM - 1]);
    }
  }
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
      const double s = ((double)pos[3 * i + a] - g.o[a]) * g.inv_h;
      if (!(fabs(s) < 1e15)) { ok = false; bidx[a] = 0; continue; }
      const long long f = (long long)floor(s);
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

// coefficient * w^power per particle; coef_kind: 0 -> 1, 1 -> -alpha, 2 -> +alpha^2
template <typename P, typename R>
__global__ void k_scatter(const P* __restrict__ pos, const P* __restrict__ w, int64_t n, int power,
                          int coef_kind, const double* __restrict__ sc, const int* __restrict__ brick,
                          const int* __restrict__ rank, const int* __restrict__ start,
                          typename RecOf<R>::type* __restrict__ rec) {
  double coef = 1.0;
  if (coef_kind == 1) coef = -sc[SC_ALPHA];
  if (coef_kind == 2) coef = sc[SC_ALPHA] * sc[SC_ALPHA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int b = brick[i];
    if (b < 0) continue;
    const double wi = w ? (double)w[i] : 1.0;
    const double wc = coef * (power == 2 ? wi * wi : wi);
    typename RecOf<R>::type r;
    r.x = (R)pos[3 * i];
    r.y = (R)pos[3 * i + 1];
    r.z = (R)pos[3 * i + 2];
    r.w = (R)wc;
    rec[start[b] + rank[i]] = r;
  }
}

// Per-axis taps: up to 3 (TSC) or 2 (CIC) cells relative to the tile, with weights.
template <int ASSIGN, typename T>
__device__ __forceinline__ void axis_taps(double s, long long fbase, int tile0, int* idx, T* wt) {
  if (ASSIGN == 2) {
    const double i0 = floor(s);
    const T d = (T)(s - i0);
    const int rel = (int)((long long)i0 - fbase) + tile0;
    idx[0] = rel; wt[0] = T(1) - d;
    idx[1] = rel + 1; wt[1] = d;
  } else {
    const double i0 = floor(s + 0.5);
    const T d = (T)(s - i0);
    const int rel = (int)((long long)i0 - fbase) + tile0;
    const T a = T(0.5) - d, b = T(0.5) + d;
    idx[0] = rel - 1; wt[0] = T(0.5) * a * a;
    idx[1] = rel; wt[1] = T(0.75) - d * d;
    idx[2] = rel + 1; wt[2] = T(0.5) * b * b;
  }
}

template <int ASSIGN, typename R, typename T>
__global__ void k_paint_brick(const typename RecOf<R>::type* __restrict__ rec, const int* __restrict__ start,
                              const int* __restrict__ count, PaintGeo g, int nphase, const double* __restrict__ sc,
                              int maxw_slot, T* __restrict__ tiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* acc = reinterpret_cast<long long*>(smem_raw);
  const int ts3 = g.ts * g.ts * g.ts;
  const int b = blockIdx.x;
  const int bx = b % g.nb, by = (b / g.nb) % g.nb, bz = b / (g.nb * g.nb);
  for (int i = threadIdx.x; i < nphase * ts3; i += blockDim.x) acc[i] = 0;
  const int cnt = count[b];
  // fixed-point scale 2^e with cnt * max|w| * 2^e < 2^61 (no overflow of the tile sums)
  const double bound = (double)cnt * sc[maxw_slot];
  int ex = 0;
  if (bound > 0) frexp(bound, &ex);
  const int e = 61 - ex;
  const double scale = ldexp(1.0, e);
  __syncthreads();
  const int beg = start[b];
  constexpr int NT = ASSIGN == 2 ? 2 : 3;
  for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
    const typename RecOf<R>::type r = rec[beg + k];
    const double p3[3] = {(double)r.x, (double)r.y, (double)r.z};
    const int borg[3] = {bx * g.bs, by * g.bs, bz * g.bs};
    double s[3];
    long long fb[3];
    int t0[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s[a] = (p3[a] - g.o[a]) * g.inv_h;
      fb[a] = (long long)floor(s[a]);
      t0[a] = (int)(wrapi(fb[a], g.n) - borg[a]) + 1;
    }
    const T wgt = (T)r.w;
    for (int ph = 0; ph < nphase; ++ph) {
      int ix[NT], iy[NT], iz[NT];
      T wx[NT], wy[NT], wz[NT];
      const double sh = ph ? 0.5 : 0.0;
      axis_taps<ASSIGN, T>(s[0] + sh, fb[0], t0[0], ix, wx);
      axis_taps<ASSIGN, T>(s[1] + sh, fb[1], t0[1], iy, wy);
      axis_taps<ASSIGN, T>(s[2] + sh, fb[2], t0[2], iz, wz);
      long long* a = acc + ph * ts3;
#pragma unroll
      for (int c = 0; c < NT; ++c) {
#pragma unroll
        for (int bb = 0; bb < NT; ++bb) {
          const T wzy = wgt * wz[c] * wy[bb];
          const int rowoff = (iz[c] * g.ts + iy[bb]) * g.ts;
#pragma unroll
          for (int aa = 0; aa < NT; ++aa) {
            const double v = (double)(wzy * wx[aa]);
            const long long q = __double2ll_rn(v * scale);
            // taps stay inside the tile by construction; the guard only protects shared memory
            if ((unsigned)iz[c] < (unsigned)g.ts && (unsigned)iy[bb] < (unsigned)g.ts &&
                (unsigned)ix[aa] < (unsigned)g.ts)
              atomicAdd(reinterpret_cast<unsigned long long*>(a + rowoff + ix[aa]),
                        static_cast<unsigned long long>(q));
          }
        }
      }
    }
  }
  __syncthreads();
  const double inv = ldexp(1.0, -e);
  for (int i = threadIdx.x; i < nphase * ts3; i += blockDim.x) {
    const int ph = i / ts3, j = i % ts3;
    tiles[((size_t)b * nphase + ph) * ts3 + j] = (T)((double)acc[i] * inv);
  }
}

template <typename T>
__global__ void k_fold(const T* __restrict__ tiles, PaintGeo g, int nphase, const double* __restrict__ sc,
                       int subtract_mean, T* __restrict__ mesh_a, T* __restrict__ mesh_b) {
  const int n = g.n;
  const int64_t ncell = (int64_t)n * n * n;
  const int ts = g.ts, ts3 = ts * ts * ts;
  const double mean = subtract_mean ? sc[SC_SUMWG] / (double)ncell : 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(c % n), y = (int)((c / n) % n), z = (int)(c / ((int64_t)n * n));
    const int cc[3] = {x, y, z};
    int nd[3], db[3][2], dt[3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int B = cc[a] / g.bs, l = cc[a] % g.bs;
      int k = 0;
      // tile of brick B covers cells [bs*B - 1, bs*B + bs + 2]
      if (l <= 2) { db[a][k] = (B - 1 + g.nb) % g.nb; dt[a][k] = l + g.bs + 1; ++k; }
      db[a][k] = B; dt[a][k] = l + 1; ++k;
      if (l == g.bs - 1 && k < 2) { db[a][k] = (B + 1) % g.nb; dt[a][k] = 0; ++k; }
      nd[a] = k;
    }
    for (int ph = 0; ph < nphase; ++ph) {
      double v = 0.0;
      for (int iz = 0; iz < nd[2]; ++iz)
        for (int iy = 0; iy < nd[1]; ++iy)
          for (int ix = 0; ix < nd[0]; ++ix) {
            const int b = (db[2][iz] * g.nb + db[1][iy]) * g.nb + db[0][ix];
            const int j = (dt[2][iz] * ts + dt[1][iy]) * ts + dt[0][ix];
            v += (double)tiles[((size_t)b * nphase + ph) * ts3 + j];
          }
      (ph ? mesh_b : mesh_a)[c] = (T)(v - mean);
    }
  }
}

template <typename P>
npc_status paint_count(npc_ctx* ctx, const DevCatalog& c, const PaintGeo& g, int* count, int* brick,
                       int* rank) {
  if (c.n == 0) return NPC_OK;
  const int blocks = (int)std::min<int64_t>((c.n + 255) / 256, (int64_t)ctx->num_sms * 16);
  k_brick_count<P><<<blocks, 256, 0, ctx->stream>>>((const P*)c.pos, c.n, g, count, brick, rank);
  NPC_LAUNCH(ctx);
  return NPC_OK;
}

template <typename P, typename R>
npc_status paint_scatter(npc_ctx* ctx, const DevCatalog& c, int power, int coef_kind, const double* sc,
                         const int* brick, const int* rank, const int* start, void* rec) {
  if (c.n == 0) return NPC_OK;
  const int blocks = (int)std::min<int64_t>((c.n + 255) / 256, (int64_t)ctx->num_sms * 16);
  k_scatter<P, R><<<blocks, 256, 0, ctx->stream>>>((const P*)c.pos, (const P*)c.w, c.n, power, coef_kind,
                                                   sc, brick, rank, start,
                                                   (typename RecOf<R>::type*)rec);
  NPC_LAUNCH(ctx);
  return NPC_OK;
}

template <typename R, typename T>
npc_status paint_impl(npc_ctx* ctx, const DevCatalog& d, const DevCatalog* r, const npc_mesh_spec& m,
                      int weight_power, const double* sc, void* mesh_a, void* mesh_b) {
  PaintGeo g;
  g.n = m.n;
  g.bs = m.n >= 64 ? 16 : m.n / 4;
  g.nb = m.n / g.bs;
  g.ts = g.bs + 4;
  for (int a = 0; a < 3; ++a) g.o[a] = m.origin[a];
  g.inv_h = (double)m.n / m.box;
  const int nphase = m.interlace ? 2 : 1;
  const int nbricks = g.nb * g.nb * g.nb;
  const int64_t ntot = d.n + (r ? r->n : 0);
  int *count, *start, *brick, *rank;
  void* rec;
  void* tiles;
  const size_t ts3 = (size_t)g.ts * g.ts * g.ts;
  NPC_TRY(ws_get(ctx, "paint.count", sizeof(int) * nbricks, (void**)&count));
  NPC_TRY(ws_get(ctx, "paint.start", sizeof(int) * nbricks, (void**)&start));
  NPC_TRY(ws_get(ctx, "paint.brick", sizeof(int) * std::max<int64_t>(ntot, 1), (void**)&brick));
  NPC_TRY(ws_get(ctx, "paint.rank", sizeof(int) * std::max<int64_t>(ntot, 1), (void**)&rank));
  NPC_TRY(ws_get(ctx, "paint.rec", sizeof(typename RecOf<R>::type) * std::max<int64_t>(ntot, 1), &rec));
  NPC_TRY(ws_get(ctx, "paint.tiles", sizeof(T) * ts3 * nbricks * nphase, &tiles));
  NPC_CUDA(ctx, cudaMemsetAsync(count, 0, sizeof(int) * nbricks, ctx->stream));
  const bool dd = d.dtype == 1;
  // counting: data then randoms share the brick counters (ranks continue)
  if (dd) NPC_TRY(paint_count<double>(ctx, d, g, count, brick, rank));
  else NPC_TRY(paint_count<float>(ctx, d, g, count, brick, rank));
  if (r) {
    if (r->dtype == 1) NPC_TRY(paint_count<double>(ctx, *r, g, count, brick + d.n, rank + d.n));
    else NPC_TRY(paint_count<float>(ctx, *r, g, count, brick + d.n, rank + d.n));
  }
  k_scan<<<1, 1024, 0, ctx->stream>>>(count, nbricks, start);
  NPC_LAUNCH(ctx);
  if (dd) NPC_TRY((paint_scatter<double, R>(ctx, d, weight_power, 0, sc, brick, rank, start, rec)));
  else NPC_TRY((paint_scatter<float, R>(ctx, d, weight_power, 0, sc, brick, rank, start, rec)));
  if (r) {
    const int kind = weight_power == 1 ? 1 : 2;
    if (r->dtype == 1)
      NPC_TRY((paint_scatter<double, R>(ctx, *r, weight_power, kind, sc, brick + d.n, rank + d.n, start, rec)));
    else
      NPC_TRY((paint_scatter<float, R>(ctx, *r, weight_power, kind, sc, brick + d.n, rank + d.n, start, rec)));
  }
  const size_t smem = sizeof(long long) * ts3 * nphase;
  const int slot = weight_power == 1 ? SC_MAXW_F : SC_MAXW_N;
  if (m.assign == 2) {
    auto kern = k_paint_brick<2, R, T>;
    NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<nbricks, 256, smem, ctx->stream>>>((const typename RecOf<R>::type*)rec, start, count, g, nphase, sc,
                                              slot, (T*)tiles);
  } else {
    auto kern = k_paint_brick<3, R, T>;
    NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<nbricks, 256, smem, ctx->stream>>>((const typename RecOf<R>::type*)rec, start, count, g, nphase, sc,
                                              slot, (T*)tiles);
  }
  NPC_LAUNCH(ctx);
  const int64_t ncell = (int64_t)m.n * m.n * m.n;
  const int fblocks = (int)std::min<int64_t>((ncell + 255) / 256, (int64_t)ctx->num_sms * 32);
  const int sub = (m.periodic && weight_power == 1) ? 1 : 0;
  k_fold<T><<<fblocks, 256, 0, ctx->stream>>>((const T*)tiles, g, nphase, sc, sub, (T*)mesh_a, (T*)mesh_b);
  NPC_LAUNCH(ctx);
  return NPC_OK;
}

}  // namespace

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
  if (prec == NPC_PREC_FP64) return paint_impl<double, double>(ctx, d, r, m, weight_power, dev_scalars, mesh_a, mesh_b);
  if (any_double) return paint_impl<double, float>(ctx, d, r, m, weight_power, dev_scalars, mesh_a, mesh_b);
  return paint_impl<float, float>(ctx, d, r, m, weight_power, dev_scalars, mesh_a, mesh_b);
}
