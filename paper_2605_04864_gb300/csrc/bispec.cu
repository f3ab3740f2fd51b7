// Bispectrum multipoles: Scoccimarro B_l (Sec. 2.2, Eq. bi_sco) with l on the first (smallest)
// side, the compressed TripoSH multipoles B_l0l (Sec. 4, Eq. new_bispec) and their analytic shot
// noise (Sec. 5.4), for a periodic box with a global line of sight.
//
// Pipeline (all bins resident in HBM):
//   1. forward transforms of the FKP field and of the w^2 N-field (power.cu passes, kz pruned to
//      the sphere |q| <= 2 k_max that the closure can reach);
//   2. k_fft_x_combine: last forward pass + interlacing + window compensation -> X_0(q), N_0(q);
//   3. k_bin_cross: shell sums of Re[X_0 N_0^*] L_l(mu) and of L_l(mu) on the k-bins and on the
//      unit-width shells of the k_3 compression (shot-noise ingredients H_l, Q_l, N_mode);
//   4. shell-filtered inverse transforms F_b(x) = sum_{q in b} X(q) e^{iq.x} for F_0 (X_0), F_2
//      (L_2(mu) X_0), the indicator I_b (1 per mode, for the triangle counts) and the full fields
//      G^(l) = sum_{|q| <= 2k_max} L_l(mu) X_0(q) e^{iq.x}: x rows only inside the sphere
//      (k_shell_x), y columns from the compact rows (k_shell_y), z columns of two real fields at
//      a time as one complex inverse transform (k_shell_z);
//   5. k_triple: sum_x F_i F_j F_k for every (i <= j, k) and sum_x F_i F_j G^(l) -- float products
//      over cells staged in shared memory, float64 accumulation per chunk of cells, per-CTA
//      partials reduced in a fixed order;
//   6. k_bispec_finalize: normalisation (2l+1)/(I33 N_T) and (2l+1)/(I33 N_i N_j), shot noise.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "fft_core.cuh"

namespace {

constexpr int BT = 256;

template <typename T>
__device__ __forceinline__ T sinc_p(T a, int p) {
  const T s = a == T(0) ? T(1) : sin(a) / a;
  T r = s;
  for (int i = 1; i < p; ++i) r *= s;
  return r;
}

// ------------------------------------------------------------------------------------------
// 2. last forward pass along x with interlacing and compensation
//    half[f][kz][ky][kx] (KZ planes; fields ordered phase a, phase b per output)
//    -> X[o][kz][ky][kx] for kz < KZ, |ky| <= KY
// ------------------------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(BT)
k_fft_x_combine(const cplx<T>* __restrict__ half, int nout, int nphase, int KZ, int KY, int assign,
                const cplx<T>* __restrict__ tw_g, cplx<T>* __restrict__ X) {
  using C = cplx<T>;
  constexpr int TPF = N / 8;
  constexpr int G = BT / TPF > 0 ? BT / TPF : 1;
  constexpr int NP = row_pad_len<N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* phs = tw + N;
  C* rows = phs + N;
  const int nf = nout * nphase;
  T* winv = reinterpret_cast<T*>(rows + (size_t)(nf + RowGroups<N, BT>::NBUF) * NP);
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += blockDim.x) {
    tw[i] = tw_g[i];
    const T a = T(M_PI) * T(i - N / 2) / T(N);
    phs[i] = cmk(cos(a), sin(a));
  }
  for (int i = tid; i <= N / 2; i += blockDim.x) winv[i] = T(1) / sinc_p<T>(T(M_PI) * T(i) / T(N), assign);
  __syncthreads();
  const int g = tid / TPF, t = tid % TPF;
  const int nyr = 2 * KY + 1;
  const int nrows = KZ * nyr;
  const size_t fstride = (size_t)KZ * N * N;
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int kz = r / nyr;
    const int jy = r % nyr - KY;
    const int ky = jy < 0 ? jy + N : jy;
    for (int f0 = 0; f0 < nf; f0 += G) {
      const int f = f0 + g;
      const bool live = g < G && f < nf;
      C v[8];
      if (live) {
        const C* src = half + (size_t)f * fstride + ((size_t)kz * N + ky) * N;
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = src[t + q * TPF];
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = cmk(T(0), T(0));
      }
      RowView<C> rv{rows + (size_t)(live ? f : nf + g) * NP};
      fft_block<N, -1>(v, t, tw, rv, RowSync<N, BT>::make(g));
      if (live) {
#pragma unroll
        for (int q = 0; q < 8; ++q) rv.st(t + q * TPF, v[q]);
      }
    }
    __syncthreads();
    for (int kx = tid; kx < N; kx += blockDim.x) {
      const int i = kx < N / 2 ? kx : kx - N;
      const int ai = i < 0 ? -i : i, aj = jy < 0 ? -jy : jy;
      const T iw = winv[ai] * winv[aj] * winv[kz];
      const int jp = RowView<C>::idx(kx);
      for (int o = 0; o < nout; ++o) {
        C x = rows[(size_t)(o * nphase) * NP + jp];
        if (nphase == 2) {
          const C ph = cmul(cmul(phs[i + N / 2], phs[jy + N / 2]), phs[kz + N / 2]);
          x = cscale(cadd(x, cmul(ph, rows[(size_t)(o * nphase + 1) * NP + jp])), T(0.5));
        }
        X[(size_t)o * fstride + ((size_t)kz * N + ky) * N + kx] = cscale(x, iw);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// 2b. survey geometry with the line of sight to each grid point: the x pass assembles X_0 and the
//     Yamamoto fields (Eq. hand with the m < 0 terms folded onto m > 0)
//       X_l = 4 pi/(2l+1) [Y_l0 A_l0 + 2 sum_{m>=1} (Re Y_lm A_lm + Im Y_lm B_lm)]   (khat at the mode)
//     for l = 1, 2, 3 (each when its output is given), from the Y_lm-weighted fields of the
//     forward plan, interlaced and compensated.  A_lm, B_lm are the transforms of Re and Im of
//     F Y_lm(xhat); X_l(-q) = (-1)^l X_l(q)^*.  Components c (l, m, part) list their phase-a field
//     ia[c] and phase-b field ib[c] (unused without interlacing).  With `comps` given the kernel
//     stores every component's interlaced, compensated spectrum there instead (component c at
//     comps + c KZ N^2): the y_L^M-weighted parts of the TripoSH field G_L^M.
// ------------------------------------------------------------------------------------------
constexpr int YAM_MAXC = 25;   // F and the parts of Y_lm, l <= 4: 1 + 3 + 5 + 7 + 9
struct YamComps {
  int nf, nc;
  int8_t l[YAM_MAXC], m[YAM_MAXC], part[YAM_MAXC];
  int8_t ia[YAM_MAXC], ib[YAM_MAXC];
};

template <typename T, int N>
__global__ void __launch_bounds__(BT)
k_fft_x_assemble_yam(const cplx<T>* __restrict__ half, int nphase, int KZ, int KY, int assign, const YNorm nrm,
                     const YamComps cp, const cplx<T>* __restrict__ tw_g, cplx<T>* __restrict__ X0o,
                     cplx<T>* __restrict__ X1o, cplx<T>* __restrict__ X2o, cplx<T>* __restrict__ X3o,
                     cplx<T>* __restrict__ comps) {
  using C = cplx<T>;
  constexpr int TPF = N / 8;
  constexpr int G = BT / TPF > 0 ? BT / TPF : 1;
  constexpr int NP = row_pad_len<N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* phs = tw + N;
  C* rows = phs + N;   // [nf + NBUF][NP]
  T* winv = reinterpret_cast<T*>(rows + (size_t)(cp.nf + RowGroups<N, BT>::NBUF) * NP);
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += blockDim.x) {
    tw[i] = tw_g[i];
    const T a = T(M_PI) * T(i - N / 2) / T(N);
    phs[i] = cmk(cos(a), sin(a));
  }
  for (int i = tid; i <= N / 2; i += blockDim.x) winv[i] = T(1) / sinc_p<T>(T(M_PI) * T(i) / T(N), assign);
  __syncthreads();
  const int g = tid / TPF, t = tid % TPF;
  const int nyr = 2 * KY + 1;
  const int nrows = KZ * nyr;
  const size_t fstride = (size_t)KZ * N * N;
  C* outs[4] = {X0o, X1o, X2o, X3o};
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int kz = r / nyr;
    const int jy = r % nyr - KY;
    const int ky = jy < 0 ? jy + N : jy;
    for (int f0 = 0; f0 < cp.nf; f0 += G) {
      const int f = f0 + g;
      const bool live = g < G && f < cp.nf;
      C v[8];
      if (live) {
        const C* src = half + (size_t)f * fstride + ((size_t)kz * N + ky) * N;
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = src[t + q * TPF];
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = cmk(T(0), T(0));
      }
      RowView<C> rv{rows + (size_t)(live ? f : cp.nf + g) * NP};
      fft_block<N, -1>(v, t, tw, rv, RowSync<N, BT>::make(g));
      if (live) {
#pragma unroll
        for (int q = 0; q < 8; ++q) rv.st(t + q * TPF, v[q]);
      }
    }
    __syncthreads();
    for (int kx = tid; kx < N; kx += blockDim.x) {
      const int i = kx < N / 2 ? kx : kx - N;
      const int ai = i < 0 ? -i : i, aj = jy < 0 ? -jy : jy;
      const T iw = winv[ai] * winv[aj] * winv[kz];
      const int jp = RowView<C>::idx(kx);
      const C ph = cmul(cmul(phs[i + N / 2], phs[jy + N / 2]), phs[kz + N / 2]);
      const T fi = T(i), fj = T(jy), fk = T(kz);
      const T r2 = fi * fi + fj * fj + fk * fk;
      const T inv = r2 > T(0) ? rsqrt(r2) : T(0);
      const T ux = fi * inv, uy = fj * inv, uz = r2 > T(0) ? fk * inv : T(1);
      C acc[4] = {cmk(T(0), T(0)), cmk(T(0), T(0)), cmk(T(0), T(0)), cmk(T(0), T(0))};
      const size_t o = ((size_t)kz * N + ky) * N + kx;
      for (int c = 0; c < cp.nc; ++c) {
        C x = rows[(size_t)cp.ia[c] * NP + jp];
        if (nphase == 2) x = cscale(cadd(x, cmul(ph, rows[(size_t)cp.ib[c] * NP + jp])), T(0.5));
        x = cscale(x, iw);
        if (comps) {
          comps[(size_t)c * fstride + o] = x;
          continue;
        }
        const int l = cp.l[c];
        if (l == 0) {
          acc[0] = x;
          continue;
        }
        T yr, yi;
        ylm_eval<T>(l, cp.m[c], ux, uy, uz, nrm, yr, yi);
        const T wgt = cp.m[c] == 0 ? yr : T(2) * (cp.part[c] == PART_IM ? yi : yr);
        acc[l] = cadd(acc[l], cscale(x, wgt));
      }
      if (comps) continue;
      X0o[o] = acc[0];
#pragma unroll
      for (int l = 1; l <= 3; ++l)
        if (outs[l]) outs[l][o] = cscale(acc[l], T(4.0 * M_PI) / T(2 * l + 1));
    }
    __syncthreads();
  }
}

// Catalogue moments of the survey self term: c_p Y_2m(xhat_p) for m = 0, 1, 2 as five reals
// (Y_20, Re Y_21, Im Y_21, Re Y_22, Im Y_22), c_p = w_p^3, per-block float64 partials in a fixed
// order; xhat_p from the observer.
constexpr int YM_BLOCKS = 512, YM_THREADS = 256;
template <typename P>
__global__ void __launch_bounds__(YM_THREADS)
k_cat_ylm2(const P* __restrict__ pos, const P* __restrict__ w, int64_t n, double ox, double oy, double oz,
           const YNorm nrm, double* __restrict__ part) {
  __shared__ double sh[5][YM_THREADS];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(n, beg + chunk);
  double a[5] = {0, 0, 0, 0, 0};
  const double n20 = nrm.v[3], n21 = nrm.v[4], n22 = nrm.v[5];
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
    const double x = (double)pos[3 * i] - ox, y = (double)pos[3 * i + 1] - oy, z = (double)pos[3 * i + 2] - oz;
    const double r2 = x * x + y * y + z * z;
    if (!(r2 > 0)) continue;
    const double inv = 1.0 / sqrt(r2);
    const double ux = x * inv, uy = y * inv, uz = z * inv;
    const double wi = w ? (double)w[i] : 1.0;
    const double c = wi * wi * wi;
    a[0] += c * n20 * (1.5 * uz * uz - 0.5);
    a[1] += c * n21 * (-3.0 * uz) * ux;
    a[2] += c * n21 * (-3.0 * uz) * uy;
    a[3] += c * n22 * 3.0 * (ux * ux - uy * uy);
    a[4] += c * n22 * 3.0 * (2.0 * ux * uy);
  }
  for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = a[k];
  __syncthreads();
  for (int off = YM_THREADS / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off)
      for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x < 5) part[blockIdx.x * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

// C_2m = data sums - alpha^3 random sums, fixed order (one warp)
__global__ void k_cat_ylm2_final(const double* __restrict__ pd, const double* __restrict__ pr, int nblk,
                                 int have_randoms, const double* __restrict__ sc, double* __restrict__ mom) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  double d[5] = {0, 0, 0, 0, 0}, r[5] = {0, 0, 0, 0, 0};
  for (int b = lane; b < nblk; b += 32)
    for (int k = 0; k < 5; ++k) {
      d[k] += pd[b * 5 + k];
      if (have_randoms) r[k] += pr[b * 5 + k];
    }
  for (int k = 0; k < 5; ++k)
    for (int off = 16; off > 0; off >>= 1) {
      d[k] += __shfl_down_sync(0xffffffffu, d[k], off);
      r[k] += __shfl_down_sync(0xffffffffu, r[k], off);
    }
  if (lane == 0) {
    const double a = sc[SC_ALPHA];
    for (int k = 0; k < 5; ++k) mom[k] = d[k] - a * a * a * r[k];
  }
}

// ------------------------------------------------------------------------------------------
// Warp-segmented accumulation of NS sums into per-warp float64 partials (runs of consecutive
// lanes with equal bin; deterministic for a fixed thread-to-mode map).
// ------------------------------------------------------------------------------------------
template <typename T, int NS>
__device__ __forceinline__ void seg_accumulate(int lane, int bin, const T (&vals)[NS], double* mypart) {
  const int pb = __shfl_up_sync(0xffffffffu, bin, 1);
  const bool head = (lane == 0) || (pb != bin);
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  const int seg = __popc(heads & (0xffffffffu >> (31 - lane)));
  unsigned addm = 0;
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int off = 1 << st;
    const int os = __shfl_up_sync(0xffffffffu, seg, off);
    if (lane >= off && os == seg) addm |= 1u << st;
  }
  const bool last = (lane == 31) || ((heads >> (lane + 1)) & 1u);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    T x = vals[s];
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const T y = __shfl_up_sync(0xffffffffu, x, 1 << st);
      if (addm & (1u << st)) x += y;
    }
    if (last && bin >= 0) atomicAdd(mypart + (size_t)bin * NS + s, (double)x);
  }
}

// ------------------------------------------------------------------------------------------
// 3. shell sums for the shot noise: per bin [sum w Re(X N*), sum w L2 Re(X N*), sum w, sum w L2]
//    on two bin sets (the k-bins and the unit-width k3 shells), modes with |ky|, kz <= KY.
// ------------------------------------------------------------------------------------------
constexpr int NCROSS = 4;
// with the TripoSH shot noise: also w L_l Re X_0 N_0^*, w L_l for l = 4, 6, 8 at 4 + 2 (l/2 - 2) + {0, 1}
constexpr int NCROSS_S = 10;

template <typename T, int N, int NC = NCROSS>
__global__ void __launch_bounds__(BT)
k_bin_cross(const cplx<T>* __restrict__ X0, const cplx<T>* __restrict__ XN, int KZ, int KY, double lx, double ly,
            double lz, const int16_t* __restrict__ tab_m, int nbm, const int16_t* __restrict__ tab_q, int nbq,
            int n2max, double* __restrict__ part_m, double* __restrict__ part_q) {
  using C = cplx<T>;
  constexpr int NW = BT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* pm = part_m + ((size_t)blockIdx.x * NW + warp) * nbm * NC;
  double* pq = part_q + ((size_t)blockIdx.x * NW + warp) * nbq * NC;
  const int nyr = 2 * KY + 1;
  const int nrows = (KY + 1) * nyr;
  const size_t fstride = (size_t)KZ * N * N;
  (void)fstride;
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int kz = r / nyr;
    const int jy = r % nyr - KY;
    const int ky = jy < 0 ? jy + N : jy;
    for (int jb = warp * 32; jb < N; jb += blockDim.x) {
      const int j = jb + lane;
      const int i = j < N / 2 ? j : j - N;
      const int n2 = i * i + jy * jy + kz * kz;
      int bm = -1, bq = -1;
      T vals[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) vals[q] = T(0);
      if (j < N && n2 > 0 && n2 <= n2max && i != -N / 2 && jy != -N / 2) {
        bm = tab_m[n2];
        bq = tab_q[n2];
        const size_t idx = ((size_t)kz * N + ky) * N + j;
        const C a = X0[idx], b = XN[idx];
        const T cr = a.x * b.x + a.y * b.y;
        const T kk = sqrt(T(n2));
        const T mu = (T(i) * T(lx) + T(jy) * T(ly) + T(kz) * T(lz)) / kk;
        const T l2 = T(1.5) * mu * mu - T(0.5);
        const T w = kz > 0 ? T(2) : T(1);
        vals[0] = w * cr;
        vals[1] = w * l2 * cr;
        vals[2] = w;
        vals[3] = w * l2;
        if constexpr (NC > NCROSS) {
          // L_3 .. L_8 by the three-term recurrence (l+1) L_{l+1} = (2l+1) mu L_l - l L_{l-1}
          T lm1 = mu, lc = l2;
#pragma unroll
          for (int l = 2; l < 8; ++l) {
            const T ln = (T(2 * l + 1) * mu * lc - T(l) * lm1) / T(l + 1);
            lm1 = lc;
            lc = ln;
            if (l + 1 == 4 || l + 1 == 6 || l + 1 == 8) {
              const int o = 4 + 2 * ((l + 1) / 2 - 2);
              vals[o] = w * lc * cr;
              vals[o + 1] = w * lc;
            }
          }
        }
      }
      T vm[NC], vq[NC];
#pragma unroll
      for (int s = 0; s < NC; ++s) {
        vm[s] = bm >= 0 ? vals[s] : T(0);
        vq[s] = bq >= 0 ? vals[s] : T(0);
      }
      seg_accumulate<T, NC>(lane, bm, vm, pm);
      seg_accumulate<T, NC>(lane, bq, vq, pq);
    }
  }
}

// ------------------------------------------------------------------------------------------
// 4. shell-filtered inverse transforms
// ------------------------------------------------------------------------------------------
struct ShellField {
  int8_t src;     // 0: X_0, 1: ones (indicator), 2: X_0 N_0^* (FFT-method shot noise), 3: X_2 (survey),
                  // 4: X_1, 5: X_3 (survey, odd: anti-Hermitian, taken times -i),
                  // 6: X of tracer 2, 7: X of tracer 3 (multi-tracer bispectra),
                  // 8: a stored component spectrum `comp` (TripoSH G_L^M parts, bin -1)
  int8_t mult;    // 0: 1, 1: L_yl(mu) (times -i for odd yl), 2: the TripoSH weight of (yl, ym, ypart)
  int16_t bin;    // >= 0: modes of this bin; -1: all modes with n2 <= n2cap
  int K;          // kz <= K, |ky| <= K
  int8_t yl, ym;  // mult 2: the field is a part of sum_q e^{iqx} y_l^{m*}(qhat) S(q), m >= 0, S the source
                  // (X: the TripoSH shell F_l^m; ones: its indicator for the FFT-method shot noise)
  int8_t ypart;   // mult 2: 0 its real part, 1 its imaginary part
  int8_t comp;    // src 8: index of the stored component spectrum (TripoSH G_L^M parts)
  int64_t off1;   // offset of this field in the x-pass output (complex elements)
  int64_t off2;   // offset in the y-pass output
};

// Orthonormal frame with e3 along the global line of sight; the TripoSH weights y_l^m(qhat) are
// evaluated on the components (q.e1, q.e2, q.e3).
struct LosFrame {
  double e1[3], e2[3], e3[3];
};

// power-basis coefficients of the Legendre polynomials L_0 .. L_4
__constant__ double c_legendre[5][5] = {{1.0, 0.0, 0.0, 0.0, 0.0},
                                        {0.0, 1.0, 0.0, 0.0, 0.0},
                                        {-0.5, 0.0, 1.5, 0.0, 0.0},
                                        {0.0, -1.5, 0.0, 2.5, 0.0},
                                        {0.375, 0.0, -3.75, 0.0, 4.375}};

template <typename T>
__device__ __forceinline__ T legendre_dev(int l, T mu) {
  T r = T(0);
  for (int k = l; k >= 0; --k) r = r * mu + T(c_legendre[l][k]);
  return r;
}

// Racah-normalised y_l^m = sqrt(4 pi/(2l+1)) Y_l^m for 0 <= m <= l <= 4 at the unit vector (x, y, z):
// (-1)^m sqrt((l-m)!/(l+m)!) (d^m L_l/dmu^m)(z) (x + i y)^m, the Condon-Shortley phase included.
template <typename T>
__device__ __forceinline__ void ylm_frame(int l, int m, T x, T y, T z, T& re, T& im) {
  T d = T(0), zp = T(1);
  for (int k = m; k <= l; ++k) {
    T f = T(c_legendre[l][k]);
    for (int q = k - m + 1; q <= k; ++q) f *= T(q);   // k!/(k-m)!
    d += f * zp;
    zp *= z;
  }
  double ratio = 1.0;
  for (int q = l - m + 1; q <= l + m; ++q) ratio *= q;
  const T nrm = T((m & 1) ? -1.0 : 1.0) / sqrt(T(ratio));
  T pr = T(1), pi = T(0);
  for (int q = 0; q < m; ++q) {
    const T t = pr * x - pi * y;
    pi = pr * y + pi * x;
    pr = t;
  }
  re = nrm * d * pr;
  im = nrm * d * pi;
}

// x rows: for every (kz <= Kmax, |ky| <= Kmax) row, every field whose K covers it.  The shells and
// their triple products are band-limited, so they run on a grid of NS <= n points per axis (the
// smallest with no aliasing of the closed triples); row kx' of the NS grid holds the integer
// frequency i = kx' (kx' < NS/2) or kx' - NS, read from the n-grid spectrum X0.
template <typename T, int NS, bool YW>
__global__ void __launch_bounds__(BT)
k_shell_x(const cplx<T>* __restrict__ X0, const cplx<T>* __restrict__ XN, const cplx<T>* __restrict__ X2,
          const cplx<T>* __restrict__ X1, const cplx<T>* __restrict__ X3, const cplx<T>* __restrict__ XB,
          const cplx<T>* __restrict__ XC, const cplx<T>* __restrict__ XCOMP, int KZX, int nfine,
          const ShellField* __restrict__ fields, int nfields, int Kmax, const int16_t* __restrict__ tab, int n2cap,
          const LosFrame fr, const cplx<T>* __restrict__ tw_g, cplx<T>* __restrict__ T1) {
  using C = cplx<T>;
  constexpr int TPF = NS / 8;
  constexpr int G = BT / TPF > 0 ? BT / TPF : 1;
  constexpr int NP = row_pad_len<NS>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* xrow = tw + NS;                  // X_0 row
  C* xnrow = xrow + NS;               // X_0 N_0^* row (when XN is given)
  C* x2row = xnrow + NS;              // Yamamoto X_2 row (when X2 is given)
  C* x1row = x2row + NS;              // Yamamoto X_1, X_3 rows (when given)
  C* x3row = x1row + NS;
  C* xbrow = x3row + NS;              // the X rows of tracers 2 and 3 (when given)
  C* xcrow = xbrow + NS;
  T* murow = reinterpret_cast<T*>(xcrow + NS);  // mu = qhat . los per kx
  int* binrow = reinterpret_cast<int*>(murow + NS);  // bin per kx (-1 excluded), n2 per kx
  int* n2row = binrow + NS;
  C* bufs = reinterpret_cast<C*>(n2row + NS);   // NBUF x NP
  const int tid = threadIdx.x;
  for (int i = tid; i < NS; i += blockDim.x) tw[i] = tw_g[i];
  const int g = tid / TPF, t = tid % TPF;
  const int nyr = 2 * Kmax + 1;
  const int nrows = (Kmax + 1) * nyr;
  __syncthreads();
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int kz = r / nyr;
    const int jy = r % nyr - Kmax;
    const int ky = jy < 0 ? jy + nfine : jy;
    const int ay = jy < 0 ? -jy : jy;
    for (int kx = tid; kx < NS; kx += blockDim.x) {
      const int i = kx < NS / 2 ? kx : kx - NS;
      const int fx = i < 0 ? i + nfine : i;
      const int n2 = i * i + jy * jy + kz * kz;
      const bool inrange = i != -NS / 2 && i != -nfine / 2 && jy != -nfine / 2 && n2 <= n2cap;
      const size_t src = ((size_t)kz * nfine + ky) * nfine + fx;
      xrow[kx] = (inrange && kz < KZX) ? X0[src] : cmk(T(0), T(0));
      if (XN) xnrow[kx] = (inrange && kz < KZX) ? cmul(X0[src], cconj(XN[src])) : cmk(T(0), T(0));
      if (X2) x2row[kx] = (inrange && kz < KZX) ? X2[src] : cmk(T(0), T(0));
      if (X1) x1row[kx] = (inrange && kz < KZX) ? X1[src] : cmk(T(0), T(0));
      if (X3) x3row[kx] = (inrange && kz < KZX) ? X3[src] : cmk(T(0), T(0));
      if (XB) xbrow[kx] = (inrange && kz < KZX) ? XB[src] : cmk(T(0), T(0));
      if (XC) xcrow[kx] = (inrange && kz < KZX) ? XC[src] : cmk(T(0), T(0));
      const T kk = sqrt(T(n2));
      murow[kx] = n2 > 0 ? (T(i) * T(fr.e3[0]) + T(jy) * T(fr.e3[1]) + T(kz) * T(fr.e3[2])) / kk : T(0);
      binrow[kx] = inrange ? tab[n2] : -1;
      n2row[kx] = inrange ? n2 : -1;
    }
    __syncthreads();
    // fields active on this row
    for (int f0 = 0; f0 < nfields; f0 += G) {
      const int f = f0 + g;
      bool live = g < G && f < nfields;
      ShellField sf{};
      if (live) {
        sf = fields[f];
        live = kz <= sf.K && ay <= sf.K;
      }
      C v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int kx = t + q * TPF;
        C a = cmk(T(0), T(0));
        if (live) {
          const bool in = sf.bin >= 0 ? (binrow[kx] == sf.bin) : (n2row[kx] >= 0);
          if (in) {
            switch (sf.src) {
              case 0: a = xrow[kx]; break;
              case 2: a = xnrow[kx]; break;
              case 3: a = x2row[kx]; break;
              case 4: a = x1row[kx]; break;
              case 5: a = x3row[kx]; break;
              case 6: a = xbrow[kx]; break;
              case 7: a = xcrow[kx]; break;
              case 8: {
                const int ii = kx < NS / 2 ? kx : kx - NS;
                const int fx = ii < 0 ? ii + nfine : ii;
                a = kz < KZX ? XCOMP[(size_t)sf.comp * KZX * nfine * nfine + ((size_t)kz * nfine + ky) * nfine + fx]
                             : cmk(T(0), T(0));
                break;
              }
              default: a = cmk(T(1), T(0));
            }
            if (sf.mult == 1) a = cscale(a, legendre_dev<T>(sf.yl, murow[kx]));
            // odd l: the source is anti-Hermitian, its shell field i A(x); -i X is Hermitian and
            // gives the real A (the imaginary part of the closure sum, Sec. 2.1)
            if ((sf.mult == 1 && (sf.yl & 1)) || sf.src == 4 || sf.src == 5) a = cmk(a.y, -a.x);
            // (YW: the call holds TripoSH fields; the other calls compile without this branch)
            if (YW && sf.mult == 2) {
              // F_l^m = sum_q e^{iqx} (Re y - i Im y) X: for even l the real weights Re y (real part)
              // and -Im y (imaginary part) are even in q; for odd l the parts are -i Im y X and
              // -i Re y X.  Every weighted spectrum stays Hermitian, so each part is a real field.
              const T ii = T(kx < NS / 2 ? kx : kx - NS), jj = T(jy), zz = T(kz);
              const T inv = n2row[kx] > 0 ? T(1) / sqrt(T(n2row[kx])) : T(0);
              const T ux = (ii * T(fr.e1[0]) + jj * T(fr.e1[1]) + zz * T(fr.e1[2])) * inv;
              const T uy = (ii * T(fr.e2[0]) + jj * T(fr.e2[1]) + zz * T(fr.e2[2])) * inv;
              const T uz = (ii * T(fr.e3[0]) + jj * T(fr.e3[1]) + zz * T(fr.e3[2])) * inv;
              T yr, yi;
              ylm_frame<T>(sf.yl, sf.ym, ux, uy, uz, yr, yi);
              if (sf.yl & 1) {
                const T w = sf.ypart ? yr : yi;
                a = cmk(a.y * w, -a.x * w);
              } else {
                a = cscale(a, sf.ypart ? -yi : yr);
              }
            }
          }
        }
        v[q] = a;
      }
      fft_block<NS, +1>(v, t, tw, RowView<C>{bufs + (size_t)g * NP}, RowSync<NS, BT>::make(g));
      if (live) {
        C* dst = T1 + sf.off1 + ((size_t)kz * (2 * sf.K + 1) + (jy + sf.K)) * NS;
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[t + q * TPF] = v[q];
      }
    }
    __syncthreads();
  }
}

template <int N> struct BCol {
  static constexpr int TX = N >= 512 ? 8 : 16;
  static constexpr int THREADS = TX * N / 8;
};

// y columns: plane p = (field, kz) from plane tables; input rows ky' = ky + K (|ky| <= K).
template <typename T, int N>
__global__ void __launch_bounds__(BCol<N>::THREADS)
k_shell_y(const cplx<T>* __restrict__ T1, const ShellField* __restrict__ fields, const int* __restrict__ plane_f,
          const int* __restrict__ plane_kz, const cplx<T>* __restrict__ tw_g, cplx<T>* __restrict__ T2) {
  using C = cplx<T>;
  constexpr int TX = BCol<N>::TX;
  constexpr int TPF = N / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* work = tw + N;
  const int tid = threadIdx.x;
  const int c = tid % TX, t = tid / TX;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = tw_g[i];
  const int p = blockIdx.y;
  const ShellField sf = fields[plane_f[p]];
  const int kz = plane_kz[p];
  const int x = blockIdx.x * TX + c;
  const C* src = T1 + sf.off1 + (size_t)kz * (2 * sf.K + 1) * N + x;
  C v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int yi = t + q * TPF;
    const int ky = yi < N / 2 ? yi : yi - N;
    v[q] = (ky >= -sf.K && ky <= sf.K) ? src[(size_t)(ky + sf.K) * N] : cmk(T(0), T(0));
  }
  __syncthreads();
  fft_block<N, +1>(v, t, tw, ColView<C>{work + c, TX});
  C* dst = T2 + sf.off2 + (size_t)kz * N * N + x;
#pragma unroll
  for (int q = 0; q < 8; ++q) dst[(size_t)(t + q * TPF) * N] = v[q];
}

// Float shell fields are stored chunk-interleaved: for every run of RCH = 128 cells the rows of all
// nfield fields follow each other (512 bytes each), so that the rows of consecutive fields of one
// chunk form one contiguous block (the tensor-core triple products copy each such block with one
// bulk copy).  Within its row, field f's cells are rotated by rf_rot(f) = 4 (f mod 8) places
// (16-byte units): once a block is in shared memory, reads of one cell offset from the rows of
// eight consecutive fields fall on distinct banks.  Float64 fields keep one row of ncell values per
// field.
constexpr int RCH = 128;
__host__ __device__ __forceinline__ int rf_rot(int field) { return 4 * (field & 7); }
__host__ __device__ __forceinline__ size_t rf_index(int field, int64_t cell, int nfield) {
  const uint64_t uc = (uint64_t)cell;
  return ((size_t)(uc >> 7) * nfield + field) * RCH + (size_t)(((int)(uc & (RCH - 1)) + rf_rot(field)) & (RCH - 1));
}

// largest |v| of a block's values of one field into fmax[f] (float bits of a non-negative value
// order as unsigned integers; a NaN orders above every finite value)
template <int THREADS>
__device__ __forceinline__ void block_absmax(unsigned m, unsigned* red, unsigned* fmax) {
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < THREADS / 32; ++w) m = max(m, red[w]);
    if (m > *reinterpret_cast<volatile unsigned*>(fmax)) atomicMax(fmax, m);
  }
  __syncthreads();
}

// z columns, two real fields (same K) per complex inverse transform:
// c(kz) = A(kz) + i B(kz), c(N - kz) = conj(A(kz)) + i conj(B(kz)); Re -> A(z), Im -> B(z).
// With fmax (float fields), the largest |value| of every field written is recorded there: the
// tensor-core triple products scale their f16 operands by it.
template <typename T, int N>
__global__ void __launch_bounds__(BCol<N>::THREADS)
k_shell_z(const cplx<T>* __restrict__ T2, const ShellField* __restrict__ fields, const int* __restrict__ pair_a,
          const int* __restrict__ pair_b, const int* __restrict__ out_a, const int* __restrict__ out_b,
          const cplx<T>* __restrict__ tw_g, T* __restrict__ R, int nfield, unsigned* __restrict__ fmax) {
  using C = cplx<T>;
  constexpr int TX = BCol<N>::TX;
  constexpr int TPF = N / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* work = tw + N;
  const int tid = threadIdx.x;
  const int c = tid % TX, t = tid / TX;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = tw_g[i];
  const int p = blockIdx.z;
  const int fa = pair_a[p], fb = pair_b[p];
  const ShellField sa = fields[fa];
  const int K = sa.K;
  const int y = blockIdx.y, x = blockIdx.x * TX + c;
  const size_t plane = (size_t)N * N;
  const C* A = T2 + sa.off2 + (size_t)y * N + x;
  const C* Bp = fb >= 0 ? T2 + fields[fb].off2 + (size_t)y * N + x : nullptr;
  C v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int zi = t + q * TPF;
    C val = cmk(T(0), T(0));
    if (zi <= K) {
      const C a = A[(size_t)zi * plane];
      const C b = Bp ? Bp[(size_t)zi * plane] : cmk(T(0), T(0));
      val = cmk(a.x - b.y, a.y + b.x);  // a + i b
    } else if (N - zi <= K) {
      const C a = A[(size_t)(N - zi) * plane];
      const C b = Bp ? Bp[(size_t)(N - zi) * plane] : cmk(T(0), T(0));
      val = cmk(a.x + b.y, -a.y + b.x);  // conj(a) + i conj(b)
    }
    v[q] = val;
  }
  __syncthreads();
  fft_block<N, +1>(v, t, tw, ColView<C>{work + c, TX});
  const size_t cell0 = (size_t)y * N + x;
  const bool has_b = out_b[p] >= 0;
  if constexpr (sizeof(T) == 4) {
    // rf_index with the z plane split off: N^2 is a multiple of RCH (N is a multiple of 16)
    const size_t cstride = (size_t)nfield * RCH;
    const size_t pchunks = plane / RCH;
    const int w0 = (int)(cell0 & (RCH - 1));
    const size_t c0k = cell0 / RCH;
    const int fa = out_a[p], fb = has_b ? out_b[p] : 0;
    const size_t oa = (size_t)fa * RCH + ((w0 + rf_rot(fa)) & (RCH - 1));
    const size_t ob = (size_t)fb * RCH + ((w0 + rf_rot(fb)) & (RCH - 1));
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const size_t base = ((size_t)(t + q * TPF) * pchunks + c0k) * cstride;
      R[base + oa] = v[q].x;
      if (has_b) R[base + ob] = v[q].y;
    }
  } else {
    T* ra = R + (size_t)out_a[p] * N * plane + cell0;
    T* rb = has_b ? R + (size_t)out_b[p] * N * plane + cell0 : nullptr;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const size_t zo = (size_t)(t + q * TPF) * plane;
      ra[zo] = v[q].x;
      if (rb) rb[zo] = v[q].y;
    }
  }
  if constexpr (sizeof(T) == 4) {
    if (fmax) {
      __shared__ unsigned red[BCol<N>::THREADS / 32];
      unsigned ma = 0u, mb = 0u;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        ma = max(ma, __float_as_uint(v[q].x) & 0x7fffffffu);
        mb = max(mb, __float_as_uint(v[q].y) & 0x7fffffffu);
      }
      block_absmax<BCol<N>::THREADS>(ma, red, fmax + out_a[p]);
      if (has_b) block_absmax<BCol<N>::THREADS>(mb, red, fmax + out_b[p]);
    }
  }
}

// ------------------------------------------------------------------------------------------
// 5. triple products over cells as a dense contraction on the tensor cores:
//      D[row, col] = sum_x P[row, x] C[x, col],  P[row, x] = A_i(x) B_j(x) for the pair (i, j) of the
//      row (two row families: A = F_0 or A = F_2, B = F_0), C[x, col] = F_0,k(x) for col = k < nb
//      and G^(l)(x) for the compressed estimator columns.  M = rows (<= 384 per CTA row group), N =
//      32 columns (4 tiles of 8), K = cells in steps of 8.  Operands are split into TF32 hi + lo
//      parts and multiplied as hi*hi + hi*lo + lo*hi (mma.sync m16n8k8, FP32 accumulation), which
//      keeps about 21 bits of each product; FP32 accumulators are added into FP64 every FLUSH
//      chunks and the per-CTA FP64 partials are reduced in a fixed order by the finalize kernel.
// ------------------------------------------------------------------------------------------
constexpr int NB_MAX = 24;
constexpr int TRI_CHUNK = 256;          // cells staged per chunk
constexpr int TRI_FLUSH = 16;           // chunks between FP64 flushes
constexpr int TRI_WARPS = 8;
// m tiles (16 rows) per warp, a template parameter: 1 (128 rows per CTA, 3 CTAs per SM) when the
// staged fields are few, else 2 (256 rows per CTA, 2 CTAs per SM)
constexpr int TRI_NT_MAX = 4;           // n tiles (8 cols) -> up to 32 columns (3 when <= 24 are used)
template <int MT> constexpr int tri_rows() { return TRI_WARPS * MT * 16; }
constexpr int TRI_COLS = TRI_NT_MAX * 8;
constexpr int TRI_SPAD = TRI_CHUNK + 4; // staging row stride (floats): 8 rows x 4 cells of an operand
                                        // fragment fall on 32 distinct banks

struct TripleArgs {
  int nrows;        // pair rows over all families (family f, pair p) -> row f * npair + p
  int npair;
  int ncol;         // used columns
  int nstage;       // distinct fields staged per chunk
  int stage_field[3 * NB_MAX + 8];  // R index of staged slot s
  int a_slot[4][NB_MAX];            // staged slot of A_i per family
  int b_slot[4][NB_MAX];            // staged slot of B_j per family
  int c_slot[TRI_COLS];             // staged slot of column c (-1: zero column)
  int nf_cols;                      // columns 0 .. nf_cols-1 are F_k (k = column), the rest G^(l)
  int64_t ncell;
  int nfield_r;                     // fields of the shell-field array (float layout: rf_index)
};

// v = hi + lo with hi = v truncated to the 10 explicit mantissa bits of tf32 (a bit mask) and the
// exact residual lo, which the tensor core reads truncated to tf32 as well: the product keeps about
// 21 bits (the error of lo's truncation is below 2^-21 |v|).
__device__ __forceinline__ void split_tf32(float v, uint32_t& hi, uint32_t& lo) {
  hi = __float_as_uint(v) & 0xffffe000u;
  lo = __float_as_uint(v - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// grid = (cell ranges, row groups of tri_rows<MT>()); block = TRI_WARPS warps; TRI_NT n tiles of 8
// columns (3 when the F_k and G^(l) columns fit in 24).  Rows run in the order row_pair (pairs
// sorted by their larger bin j) and are written back to their pair index.
// Fragment layouts of m16n8k8 (tf32): A a0 (row g, k t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4);
// B b0 (k t, col g), b1 (k t+4, col g); D d0, d1 (row g, cols 2t, 2t+1), d2, d3 (row g+8, ...),
// with g = lane/4 and t = lane%4.
// SK (split over cells): every warp takes the same TRI_MT m tiles (the whole row group) and its own
// TRI_CHUNK / TRI_WARPS cells of each staged chunk; the warps' FP64 sums are added in warp order at
// the end.  For products with few rows (at most 16 TRI_MT), where the row split would leave warps idle.
template <int TRI_NT, int TRI_MT, bool SK = false>
__global__ void __launch_bounds__(TRI_WARPS * 32, TRI_MT == 1 ? 3 : 2)
k_triple(const float* __restrict__ R, const TripleArgs A, const int* __restrict__ pair_ij,
         const int* __restrict__ row_pair, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* stage = reinterpret_cast<float*>(smem_raw);                               // [nstage][TRI_SPAD]
  double* dacc = reinterpret_cast<double*>(stage + (size_t)A.nstage * TRI_SPAD);  // [tid][NACC]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int rowbase = SK ? blockIdx.y * TRI_MT * 16 : blockIdx.y * tri_rows<TRI_MT>() + warp * TRI_MT * 16;
  int sa[TRI_MT][2], sb[TRI_MT][2], orow[TRI_MT][2];
#pragma unroll
  for (int mt = 0; mt < TRI_MT; ++mt) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = rowbase + mt * 16 + g + 8 * h;
      sa[mt][h] = sb[mt][h] = orow[mt][h] = -1;
      if (r < A.nrows) {
        const int fam = r / A.npair, p = row_pair[r % A.npair];
        const int pij = pair_ij[p];
        sa[mt][h] = A.a_slot[fam][pij & 0xffff];
        sb[mt][h] = A.b_slot[fam][pij >> 16];
        orow[mt][h] = fam * A.npair + p;
      }
    }
  }
  int scol[TRI_NT];
#pragma unroll
  for (int nt = 0; nt < TRI_NT; ++nt) {
    const int c = nt * 8 + g;
    scol[nt] = c < A.ncol ? A.c_slot[c] : -1;
  }
  constexpr int NACC = TRI_MT * TRI_NT * 4;
  double* myacc = dacc + (size_t)tid * NACC;
  for (int e = 0; e < NACC; ++e) myacc[e] = 0.0;
  float d[TRI_MT][TRI_NT][4];
#pragma unroll
  for (int mt = 0; mt < TRI_MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < TRI_NT; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) d[mt][nt][q] = 0.f;
  const int64_t per = ((A.ncell + gridDim.x - 1) / gridDim.x + TRI_CHUNK - 1) / TRI_CHUNK * TRI_CHUNK;
  const int64_t beg = (int64_t)blockIdx.x * per;
  const int64_t end = min(A.ncell, beg + per);
  int nchunk = 0;
  for (int64_t c0 = beg; c0 < end; c0 += TRI_CHUNK) {
    const int nc = (int)((end - c0) < (int64_t)TRI_CHUNK ? (end - c0) : (int64_t)TRI_CHUNK);
    __syncthreads();
    // one 128-cell row of a staged field per warp and step: a 16-byte load per lane, the row's
    // rotation undone on the store (nc is a multiple of RCH: ncell is)
    for (int rw = warp; rw < A.nstage * (TRI_CHUNK / RCH); rw += TRI_WARPS) {
      const int sl = rw / (TRI_CHUNK / RCH), half = rw % (TRI_CHUNK / RCH);
      const int field = A.stage_field[sl], rot = rf_rot(field);
      const int cl = (lane * 4 - rot) & (RCH - 1);   // logical cell of the lane's first value
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (half * RCH < nc)
        v = *reinterpret_cast<const float4*>(R + (((size_t)(c0 / RCH) + half) * A.nfield_r + field) * RCH + lane * 4);
      *reinterpret_cast<float4*>(stage + (size_t)sl * TRI_SPAD + half * RCH + cl) = v;
    }
    __syncthreads();
    constexpr int KPW = SK ? TRI_CHUNK / TRI_WARPS : TRI_CHUNK;   // cells of the chunk per warp
    const int kbeg = SK ? warp * KPW : 0;
    for (int kk = kbeg; kk < kbeg + KPW; kk += 8) {
      uint32_t bh[TRI_NT][2], bl[TRI_NT][2];
#pragma unroll
      for (int nt = 0; nt < TRI_NT; ++nt) {
        float v0 = 0.f, v1 = 0.f;
        if (scol[nt] >= 0) {
          const float* col = stage + (size_t)scol[nt] * TRI_SPAD + kk;
          v0 = col[t];
          v1 = col[t + 4];
        }
        split_tf32(v0, bh[nt][0], bl[nt][0]);
        split_tf32(v1, bh[nt][1], bl[nt][1]);
      }
#pragma unroll
      for (int mt = 0; mt < TRI_MT; ++mt) {
        uint32_t ah[4], al[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int h = q & 1;
          const int kc = kk + t + ((q >> 1) ? 4 : 0);
          float e = 0.f;
          if (sa[mt][h] >= 0) e = stage[(size_t)sa[mt][h] * TRI_SPAD + kc] * stage[(size_t)sb[mt][h] * TRI_SPAD + kc];
          split_tf32(e, ah[q], al[q]);
        }
#pragma unroll
        for (int nt = 0; nt < TRI_NT; ++nt) {
          mma_tf32(d[mt][nt], ah, bh[nt][0], bh[nt][1]);
          mma_tf32(d[mt][nt], ah, bl[nt][0], bl[nt][1]);
          mma_tf32(d[mt][nt], al, bh[nt][0], bh[nt][1]);
        }
      }
    }
    if (++nchunk == TRI_FLUSH || c0 + TRI_CHUNK >= end) {
      nchunk = 0;
      int e = 0;
#pragma unroll
      for (int mt = 0; mt < TRI_MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < TRI_NT; ++nt)
#pragma unroll
          for (int q = 0; q < 4; ++q, ++e) {
            myacc[e] += (double)d[mt][nt][q];
            d[mt][nt][q] = 0.f;
          }
    }
  }
  if constexpr (SK) {
    // add the warps' sums in warp order (warp 0's own sums first); warp 0 writes them
    __syncthreads();
    if (warp != 0) return;
    for (int q = 0; q < NACC; ++q) {
      double v = 0.0;
      for (int w = 0; w < TRI_WARPS; ++w) v += dacc[(size_t)(w * 32 + lane) * NACC + q];
      myacc[q] = v;
    }
  }
  // this CTA's partial sums as part[cta][row][col]
  int e = 0;
#pragma unroll
  for (int mt = 0; mt < TRI_MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < TRI_NT; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q, ++e) {
        const int r = orow[mt][q >> 1];
        const int c = nt * 8 + 2 * t + (q & 1);
        if (r >= 0 && c < A.ncol) part[((size_t)blockIdx.x * A.nrows + r) * A.ncol + c] = myacc[e];
      }
}

// Float64 path of the same contraction (precision NPC_PREC_FP64): one thread per (row, col)
// output over a range of cells; slow, exact to float64 rounding, for validation-size meshes.
__global__ void __launch_bounds__(256)
k_triple_f64(const double* __restrict__ R, const TripleArgs A, const int* __restrict__ pair_ij,
             double* __restrict__ part) {
  const int o = blockIdx.y * blockDim.x + threadIdx.x;
  if (o >= A.nrows * A.ncol) return;
  const int r = o / A.ncol, c = o % A.ncol;
  const int fam = r / A.npair, p = r % A.npair;
  const int pij = pair_ij[p];
  const int cs = A.c_slot[c];
  double acc = 0.0;
  if (cs >= 0) {
    const double* fa = R + (size_t)A.stage_field[A.a_slot[fam][pij & 0xffff]] * A.ncell;
    const double* fb = R + (size_t)A.stage_field[A.b_slot[fam][pij >> 16]] * A.ncell;
    const double* fc = R + (size_t)A.stage_field[cs] * A.ncell;
    const int64_t per = (A.ncell + gridDim.x - 1) / gridDim.x;
    const int64_t beg = (int64_t)blockIdx.x * per, end = min(A.ncell, beg + per);
    for (int64_t x = beg; x < end; ++x) acc += fa[x] * fb[x] * fc[x];
  }
  part[((size_t)blockIdx.x * A.nrows + r) * A.ncol + c] = acc;
}

#include "triple_tc.cuh"

// Orientation of a tensor-core triple-product launch (triple_tc.cuh).  Every output (family f,
// pair (i, j), column c) multiplies three staged fields A_{f,i} B_{f,j} C_c; two of them form a
// product row (M side) and the third a single-field column (N side, hi and lo interleaved).  The
// three assignments are tried and the one with the lowest cost is kept: per 16-cell k step each
// row tile takes two products of at least 46 cycles (N <= 64 costs as much as N = 16; above that
// about N / 2), and forming a row about half a cycle.
struct TcPlanHost {
  int nmrow = 0, nmcol = 0, n = 0, nt = 1, groups = 1, nsa = 2, nbuf = 3;
  size_t smem = 0;
  std::vector<int16_t> rx, ry, cz;   // staged slots, numbered by increasing field index
  std::vector<int> sfield, runs;     // field of each slot; runs of consecutive fields (first slot, length)
  std::vector<int> gidx;
  size_t o_rx = 0, o_ry = 0, o_cz = 0, o_sfield = 0, o_runs = 0, o_gidx = 0;   // offsets in the uploaded table
};

// need_pk (optional, npair x nf_cols): the outputs of the first nf_cols columns that are read later
// (1) or never (0, written as zero); columns from nf_cols on are always read.
bool plan_triple_tc(const TripleArgs& a, const int* pij, int max_smem, TcPlanHost& out,
                    const std::vector<char>* need_pk = nullptr) {
  if (a.npair <= 0 || a.nrows % a.npair != 0 || a.nstage > tc::MAX_SLOTS || a.ncell % tc::CHUNK != 0) return false;
  const int nfam = a.nrows / a.npair;
  // staged slots renumbered by increasing field index; runs of consecutive fields
  std::vector<int> order(a.nstage), pos(a.nstage);
  for (int q = 0; q < a.nstage; ++q) order[q] = q;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return a.stage_field[x] < a.stage_field[y]; });
  std::vector<int> sfield(a.nstage), runs;
  for (int q = 0; q < a.nstage; ++q) {
    pos[order[q]] = q;
    sfield[q] = a.stage_field[order[q]];
    if (q > 0 && sfield[q] == sfield[q - 1]) return false;   // a field staged twice
    if (q == 0 || sfield[q] != sfield[q - 1] + 1) {
      runs.push_back(q);
      runs.push_back(1);
    } else {
      runs.back() += 1;
    }
  }
  auto slot = [&](int x) { return x < 0 ? -1 : pos[x]; };
  double best = 1e300;
  bool found = false;
  for (int orient = 0; orient < 3; ++orient) {
    std::map<std::pair<int, int>, int> rows;
    std::map<int, int> cols;
    auto roles = [&](int f, int p, int c, int& u, int& v, int& w) {
      const int xa = slot(a.a_slot[f][pij[p] & 0xffff]), xb = slot(a.b_slot[f][pij[p] >> 16]), xc = slot(a.c_slot[c]);
      if (orient == 0) { u = xa; v = xb; w = xc; }
      else if (orient == 1) { u = xb; v = xc; w = xa; }
      else { u = xa; v = xc; w = xb; }
      if (u > v) std::swap(u, v);
    };
    auto needed = [&](int p, int c) {
      return a.c_slot[c] >= 0 && (!need_pk || c >= a.nf_cols || (*need_pk)[(size_t)p * a.nf_cols + c]);
    };
    for (int f = 0; f < nfam; ++f)
      for (int p = 0; p < a.npair; ++p)
        for (int c = 0; c < a.ncol; ++c) {
          if (!needed(p, c)) continue;
          int u, v, w;
          roles(f, p, c, u, v, w);
          if (u < 0 || w < 0) return false;
          rows.emplace(std::make_pair(u, v), 0);
          cols.emplace(w, 0);
        }
    const int nr = (int)rows.size(), nc = (int)cols.size();
    if (nr == 0 || nc == 0) return false;
    const int n = std::max(16, (2 * nc + 15) / 16 * 16);
    if (n > tc::MAXN) continue;
    const int tiles = (nr + 127) / 128;
    // row tiles per CTA: the most (up to three) that leave tensor memory for two stages in flight
    int nt = std::min(3, tiles), nsa = 0;
    for (; nt >= 1; --nt) {
      nsa = std::min(tc::NSA_MAX, (512 / nt - n) / tc::ACOLS);
      if (nsa >= 2) break;
    }
    if (nt < 1) continue;
    const int groups = (tiles + nt - 1) / nt;
    nt = (tiles + groups - 1) / groups;   // the same group count with the tiles spread evenly
    nsa = std::min(tc::NSA_MAX, (512 / nt - n) / tc::ACOLS);
    int nbuf = 3;
    size_t smem = tc::tc_layout(a.nstage, 3, nt, n, nc, nsa).total;
    if (smem > 200 * 1024) {
      nbuf = 2;
      smem = tc::tc_layout(a.nstage, 2, nt, n, nc, nsa).total;
    }
    if (smem > (size_t)max_smem) continue;
    const double cost = (double)tiles * 2.0 * std::max(46.0, n / 2.0) + 0.5 * nr;
    if (cost >= best) continue;
    best = cost;
    found = true;
    TcPlanHost P;
    P.sfield = sfield;
    P.runs = runs;
    P.nmrow = nr;
    P.nmcol = nc;
    P.n = n;
    P.nt = nt;
    P.groups = groups;
    P.nsa = nsa;
    P.nbuf = nbuf;
    P.smem = smem;
    int k = 0;
    for (auto& e : rows) {   // key order: rows sharing their first factor are adjacent (broadcast loads)
      e.second = k++;
      P.rx.push_back((int16_t)e.first.first);
      P.ry.push_back((int16_t)e.first.second);
    }
    k = 0;
    for (auto& e : cols) {
      e.second = k++;
      P.cz.push_back((int16_t)e.first);
    }
    P.gidx.assign((size_t)a.nrows * a.ncol, -1);
    for (int f = 0; f < nfam; ++f)
      for (int p = 0; p < a.npair; ++p)
        for (int c = 0; c < a.ncol; ++c) {
          if (!needed(p, c)) continue;
          int u, v, w;
          roles(f, p, c, u, v, w);
          P.gidx[((size_t)f * a.npair + p) * a.ncol + c] = rows.at(std::make_pair(u, v)) * nc + cols.at(w);
        }
    out = std::move(P);
  }
  return found;
}

// ------------------------------------------------------------------------------------------
// 6. normalisation and analytic shot noise (one thread per triangle / pair)
// ------------------------------------------------------------------------------------------
__device__ double g_ell_dev(int l, double t) {
  // closed forms of g_l(t) for l = 0, 2 (Appendix H, Eqs. g0, g2)
  if (l == 0) return 1.0;
  if (t == 0.0) return 0.0;
  if (t == 1.0) return 0.25;
  const double lg = log((t + 1.0) / fabs(t - 1.0));
  return (2.0 * t * (5.0 * t * t - 3.0) + 3.0 * (t * t - 1.0) * (t * t - 1.0) * lg) / (16.0 * t * t * t);
}

// Survey l = 2 shell sums: per bin [w Re X0 N0*, w Re X2 N0*, w Re X0 N2*, w, w Y_20, w Re Y_21,
// w Im Y_21, w Re Y_22, w Im Y_22] on the k-bins and on the unit-width k3 shells.
constexpr int NCS = 9;
template <typename T, int N>
__global__ void __launch_bounds__(BT)
k_bin_cross_survey(const cplx<T>* __restrict__ X0, const cplx<T>* __restrict__ X2, const cplx<T>* __restrict__ N0,
                   const cplx<T>* __restrict__ N2, int KY, const YNorm nrm, const int16_t* __restrict__ tab_m, int nbm,
                   const int16_t* __restrict__ tab_q, int nbq, int n2max, double* __restrict__ part_m,
                   double* __restrict__ part_q) {
  using C = cplx<T>;
  constexpr int NW = BT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* pm = part_m + ((size_t)blockIdx.x * NW + warp) * nbm * NCS;
  double* pq = part_q + ((size_t)blockIdx.x * NW + warp) * nbq * NCS;
  const int nyr = 2 * KY + 1;
  const int nrows = (KY + 1) * nyr;
  const T n20 = ynorm<T>(nrm, 3), n21 = ynorm<T>(nrm, 4), n22 = ynorm<T>(nrm, 5);
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int kz = r / nyr;
    const int jy = r % nyr - KY;
    const int ky = jy < 0 ? jy + N : jy;
    for (int jb = warp * 32; jb < N; jb += blockDim.x) {
      const int j = jb + lane;
      const int i = j < N / 2 ? j : j - N;
      const int n2 = i * i + jy * jy + kz * kz;
      int bm = -1, bq = -1;
      T vals[NCS];
#pragma unroll
      for (int s = 0; s < NCS; ++s) vals[s] = T(0);
      if (j < N && n2 > 0 && n2 <= n2max && i != -N / 2 && jy != -N / 2) {
        bm = tab_m[n2];
        bq = tab_q[n2];
        const size_t idx = ((size_t)kz * N + ky) * N + j;
        const C a0 = X0[idx], a2 = X2[idx], b0 = N0[idx], b2 = N2[idx];
        const T inv = rsqrt(T(n2));
        const T ux = T(i) * inv, uy = T(jy) * inv, uz = T(kz) * inv;
        const T w = kz > 0 ? T(2) : T(1);
        vals[0] = w * (a0.x * b0.x + a0.y * b0.y);
        vals[1] = w * (a2.x * b0.x + a2.y * b0.y);
        vals[2] = w * (a0.x * b2.x + a0.y * b2.y);
        vals[3] = w;
        vals[4] = w * n20 * (T(1.5) * uz * uz - T(0.5));
        vals[5] = w * n21 * T(-3) * uz * ux;
        vals[6] = w * n21 * T(-3) * uz * uy;
        vals[7] = w * n22 * T(3) * (ux * ux - uy * uy);
        vals[8] = w * n22 * T(3) * (T(2) * ux * uy);
      }
      T vm[NCS], vq[NCS];
#pragma unroll
      for (int s = 0; s < NCS; ++s) {
        vm[s] = bm >= 0 ? vals[s] : T(0);
        vq[s] = bq >= 0 ? vals[s] : T(0);
      }
      seg_accumulate<T, NCS>(lane, bm, vm, pm);
      seg_accumulate<T, NCS>(lane, bq, vq, pq);
    }
  }
}

struct FinalArgs {
  int nb, ntri, npair, nq;
  int nscoc, scoc_l[4];
  int scoc_fam[4];      // row family of each Scoccimarro multipole in the data launch partials
  int ntripo, tripo_l[2];
  int shot;
  int nparts;           // CTAs of the triple kernel
  int nrows;            // rows of the data launch partials (family * npair + pair)
  int ncol;             // columns of the data launch partials (nb F_0 columns, then G columns)
  int64_t ncell;
  double kmin, dk;
  int part_nw_cross;    // partial records of the cross-spectrum kernel
  // FFT-method shot noise (shot = 2): partials of sum_x I_a I_b G_c (family 0) and
  // sum_x I2_a I_b G_c (family 1) in s1 (columns c < nb; then, for the compressed multipoles e,
  // sum_x I_a I_b SF_e at nb + e and sum_x I_a I_b LF_e at nb + ntripo + e), of sum_x I_a I_b G2_c
  // in s2 (nb columns), of sum_x I_a G_b LF_e (family 0) and sum_x G_a I_b LF_e (family 1) in s3
  int s1_nparts, s1_nrows, s1_ncol, s2_nparts, s2_nrows, s3_nparts, s3_nrows, s3_ncol;
  int survey;           // 1: survey l = 2 shell sums (NCS per bin) and catalogue moments
  int ncs;              // sums per bin in cross_m / cross_q
  int ntri_blocks;      // leading 32-thread blocks that take the triangles (then one per pair)
};

__global__ void k_bispec_finalize(const int* __restrict__ tri, const int* __restrict__ pair_ij,
                                  const double* __restrict__ part_main, const double* __restrict__ nt_sums,
                                  const double* __restrict__ cross_m, const double* __restrict__ cross_q,
                                  const double* __restrict__ mom, const double* __restrict__ part_s1,
                                  const double* __restrict__ part_s2, const double* __restrict__ part_s3,
                                  const double* __restrict__ nt2_sums, const FinalArgs F,
                                  const double* __restrict__ sc, double* __restrict__ out) {
  const int nb = F.nb;
  const double i33 = sc[SC_I33], s3 = sc[SC_S3];
  // layout offsets
  const size_t oB = 0, oSB = (size_t)F.nscoc * F.ntri, oNT = 2 * (size_t)F.nscoc * F.ntri;
  const size_t oBB = oNT + F.ntri, oSBB = oBB + (size_t)F.ntripo * F.npair;
  const size_t oNM = oSBB + (size_t)F.ntripo * F.npair, oSC = oNM + nb;
  auto cross = [&](const double* cr, int b, int s) { return cr[(size_t)b * F.ncs + s]; };
  auto count = [&](const double* cr, int b) { return cross(cr, b, F.survey ? 3 : 2); };
  auto centre = [&](int b) { return F.kmin + (b + 0.5) * F.dk; };
  // H_l(k) = <Re X_0 N_l*> - S_l and Q_l(k) = <Re X_l N_0*> - S_l on a bin set (k-bins or k3 shells).
  // Global line of sight: both are <L_l Re X_0 N_0*> - S3 <L_l>.  Survey l = 2: the self term
  // S_2 = 4 pi/5 sum_m <Y_2m(qhat)> C_2m^* from the catalogue moments C_2m.
  auto shell_term = [&](const double* cr, int l, int b, bool q) {
    const double n = count(cr, b);
    if (n <= 0) return 0.0;
    if (l == 0) return (cross(cr, b, 0) - s3 * n) / n;
    if (!F.survey) return (cross(cr, b, 1) - s3 * cross(cr, b, 3)) / n;
    const double* c = cr + (size_t)b * F.ncs;
    const double self = 4.0 * M_PI / 5.0 * (c[4] * mom[0] + 2.0 * (c[5] * mom[1] + c[6] * mom[2] + c[7] * mom[3] +
                                                                   c[8] * mom[4]));
    return ((q ? c[1] : c[2]) - self) / n;
  };
  auto Hm = [&](int l, int b) { return shell_term(cross_m, l, b, false); };
  auto Qm = [&](int l, int b) { return shell_term(cross_m, l, b, true); };
  auto Qq = [&](int l, int b) { return shell_term(cross_q, l, b, true); };
  auto pair_index = [&](int a, int b) {   // a <= b
    int p = 0;
    for (int c = 0; c < a; ++c) p += nb - c;
    return p + b - a;
  };
  // sum over CTAs of an FFT-method partial (family fam, pair p, column c)
  auto shot_sum = [&](const double* part, int nparts, int nrows, int ncol, int fam, int p, int c) {
    double v = 0;
    for (int q = 0; q < nparts; ++q) v += part[((size_t)q * nrows + fam * F.npair + p) * ncol + c];
    return v;
  };
  auto ps1 = [&](int fam, int p, int c) { return shot_sum(part_s1, F.s1_nparts, F.s1_nrows, F.s1_ncol, fam, p, c); };
  auto ps2 = [&](int fam, int p, int c) { return shot_sum(part_s2, F.s2_nparts, F.s2_nrows, nb, fam, p, c); };
  auto ps3 = [&](int fam, int p, int c) { return shot_sum(part_s3, F.s3_nparts, F.s3_nrows, F.s3_ncol, fam, p, c); };
  // pair p (lanes of one warp): compressed multipoles and their shot noise
  auto finalize_pair = [&](int p, int lane) {
    const int i = pair_ij[p] & 0xffff, j = pair_ij[p] >> 16;
    const double ni = count(cross_m, i), nj = count(cross_m, j);
    for (int e = 0; e < F.ntripo; ++e) {
      const int l = F.tripo_l[e];
      double sg = 0;
      for (int c = 0; c < F.nparts; ++c) sg += part_main[((size_t)c * F.nrows + p) * F.ncol + nb + e];
      const double raw = (ni > 0 && nj > 0) ? (2 * l + 1) * sg / (i33 * ni * nj * (double)F.ncell) : 0.0;
      double sn = 0.0;
      if (F.shot == 2 && ni > 0 && nj > 0) {
        // FFT method: Ta + Tb + Tc - 2 S Td over the (q1, q2) pairs of the two bins
        const double ta = ps1(0, p, nb + e), td = ps1(0, p, nb + F.ntripo + e);
        const double tb = ps3(0, p, e), tc = ps3(1, p, e);
        sn = (2 * l + 1) * (ta + tb + tc - 2.0 * s3 * td) / (i33 * ni * nj * (double)F.ncell);
      } else if (F.shot && ni > 0 && nj > 0) {
        const double ci = centre(i), cj = centre(j);
        const double sgn = (l % 2) ? -1.0 : 1.0;
        double v = (l == 0 ? s3 : 0.0);
        v += sgn * g_ell_dev(l, ci / cj) * Hm(l, i);
        v += sgn * g_ell_dev(l, cj / ci) * Hm(l, j);
        // k3-shell average of Q_l over the shells the pair closes on: lanes take shells m = lane,
        // lane + 32, ..., then a fixed shuffle tree
        const double lo = fabs(ci - cj) + 0.5 * F.dk, hi = ci + cj - 0.5 * F.dk;
        double num = 0, den = 0;
        for (int m = lane; m < F.nq; m += 32) {
          const double cm = (m + 0.5) * F.dk;
          const double nm = count(cross_q, m);
          if (cm >= lo - 1e-9 * F.dk && cm <= hi + 1e-9 * F.dk && nm > 0) {
            num += nm / cm * Qq(l, m);
            den += nm / cm;
          }
        }
        for (int off = 16; off > 0; off >>= 1) {
          num += __shfl_xor_sync(0xffffffffu, num, off);
          den += __shfl_xor_sync(0xffffffffu, den, off);
        }
        if (den > 0) v += num / den;
        sn = (2 * l + 1) / i33 * v;
      }
      if (lane == 0) {
        out[oBB + (size_t)e * F.npair + p] = raw - sn;
        out[oSBB + (size_t)e * F.npair + p] = sn;
      }
    }
  };
  // blocks [0, ntb) take the triangles, one per thread; block ntb + p takes pair p as one warp
  // (FP64 arithmetic is scarce on this part, so the per-pair shell sums are spread over the lanes)
  const int ntb = F.ntri_blocks;
  if ((int)blockIdx.x >= ntb) {
    const int p = blockIdx.x - ntb, lane = threadIdx.x;
    if (p < F.npair) finalize_pair(p, lane);
    return;
  }
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = ntb * blockDim.x;
  for (int t = tid; t < F.ntri; t += nthreads) {
    const int i = tri[3 * t], j = tri[3 * t + 1], k = tri[3 * t + 2];
    const int p = pair_index(i, j);
    double sfam[4] = {0, 0, 0, 0}, snt = 0;
    for (int c = 0; c < F.nparts; ++c)
      for (int e = 0; e < F.nscoc; ++e)
        sfam[e] += part_main[((size_t)c * F.nrows + (size_t)F.scoc_fam[e] * F.npair + p) * F.ncol + k];
    snt = nt_sums[(size_t)p * nb + k];
    out[oNT + t] = snt / (double)F.ncell;
    const double ci = centre(i), cj = centre(j), ck = centre(k);
    const double c12 = (ck * ck - ci * ci - cj * cj) / (2.0 * ci * cj);
    const double c13 = (cj * cj - ci * ci - ck * ck) / (2.0 * ci * ck);
    for (int e = 0; e < F.nscoc; ++e) {
      const int l = F.scoc_l[e];
      const double raw = snt > 0 ? (2 * l + 1) * sfam[e] / (i33 * snt) : 0.0;
      double sn = 0.0;
      if (l & 1) {
        // odd multipoles: raw estimate (no shot-noise model for them)
      } else if (F.shot == 2 && snt > 0) {
        // FFT method: two-object terms T23 + T12 + T13 over the closed triplets, minus twice the
        // three-of-one-object part S N_T^(l) (each two-object term holds it once, the pure term once)
        const int pik = pair_index(i, k), pjk = pair_index(j, k);
        double tsum, ntl;
        if (l == 0) {
          tsum = ps1(0, pjk, i) + ps1(0, p, k) + ps1(0, pik, j);
          ntl = snt;
        } else {
          tsum = ps2(0, pjk, i) + ps1(1, p, k) + ps1(1, pik, j);
          ntl = nt2_sums[(size_t)p * nb + k];
        }
        sn = (2 * l + 1) * (tsum - 2.0 * s3 * ntl) / (i33 * snt);
      } else if (F.shot && snt > 0) {
        const double L12 = l == 0 ? 1.0 : 1.5 * c12 * c12 - 0.5;
        const double L13 = l == 0 ? 1.0 : 1.5 * c13 * c13 - 0.5;
        sn = (2 * l + 1) / i33 * ((l == 0 ? s3 : 0.0) + Qm(l, i) + L12 * Hm(l, j) + L13 * Hm(l, k));
      }
      out[oB + (size_t)e * F.ntri + t] = raw - sn;
      out[oSB + (size_t)e * F.ntri + t] = sn;
    }
  }
  for (int b = tid; b < nb; b += nthreads) out[oNM + b] = count(cross_m, b);
  if (tid < 8) out[oSC + tid] = sc[tid];
}

// Racah-normalised associated Legendre function cL_l^n(x): y_l^n at polar cosine x, azimuth 0
// (for n < 0, (-1)^n cL_l^{|n|})
__device__ double racah_assoc(int l, int n, double x) {
  double re, im;
  const int an = n < 0 ? -n : n;
  ylm_frame<double>(l, an, sqrt(fmax(0.0, 1.0 - x * x)), 0.0, x, re, im);
  return (n < 0 && (an & 1)) ? -re : re;
}

// per multipole: l1, l2, L, H N, then (l1 l2 L; n -n 0) for n = -4 .. 4
constexpr int SUGI_DESC = 13;
// per-bin lattice sums of the FFT-method shot noise: (Re A, Im A, Re C, Im C) for l <= 4, 0 <= m <= l
constexpr int NSB = 60;

// TripoSH multipoles from the per-combination sums red[c][i][j] = sum_x A_i(x) G(x) C_j(x) (A, C the
// parts of F_l1^m and F_l2^m of bins i and j): raw(i, j) = sum_c coef[e][c] red[c][i][j] /
// (I33 N_i N_j ncell).  shot: the analytic shot noise of Sec. 5.4, global line of sight,
//   delta_{l1 0} delta_{l2 0} delta_{L 0} S + delta_{l1 L} delta_{l2 0} (2L+1) H_L(k_i)
//   + delta_{l2 L} delta_{l1 0} (2L+1) H_L(k_j) + H N sum_m w_m q(c_i, c_j, c_m) Q_L(m) / sum_m w_m,
// all over I33, with H_L, Q_L = (sum w L_L Re X N^* - S sum w L_L) / N_mode on the k-bins and on the
// k3 shells of width dk, w_m = N_mode(m)/c_m over the shells closing the pair, and Lemma 1's
//   q(k1, k2, k3) = sum_n (-1)^n cL_l1^n(cos t13) cL_l2^{-n}(cos t23) (l1 l2 L; n -n 0).
// Output: [nmult][nb][nb] raw - shot, [nmult][nb][nb] shot, the mode counts, the scalars.
// shot = 2, the FFT method (Sec. 5.4.2): red[ncombo + c] holds the products of the indicator parts
// against the full-range X N^* field (legs 1, 2 from one object), sbins the per-bin sums A_l^m =
// sum y_l^{m*} and C_l^m = sum y_l^{m*} X N^* (legs 1, 3 and legs 2, 3 from one object, and the pure
// term): shot = [sum_c coef red_ind / ncell + H N sum_m (l1 l2 L; m -m 0) Re(A1^m C2^{-m} +
// C1^m A2^{-m} - 2 S A1^m A2^{-m})] / (I33 N_i N_j), with A^{-m} = (-1)^m conj A^m and
// C^{-m} = (-1)^{m+l} conj C^m.
__global__ void k_sugi_finalize(const double* __restrict__ red, int ncombo, const double* __restrict__ coef,
                                const double* __restrict__ desc, int nmult, int nb, const double* __restrict__ cross_m,
                                const double* __restrict__ cross_q, int nq, int ncs, int shot,
                                const double* __restrict__ sbins, double dk, double kmin,
                                const double* __restrict__ sc, double ncell, double* __restrict__ out) {
  // one warp per output (e, i, j); the lanes share the k3 shells of the ring average
  const int nn = nb * nb;
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  const double i33 = sc[SC_I33], s3 = sc[SC_S3];
  auto shell = [&](const double* cr, int L, int b) {
    const double* c = cr + (size_t)b * ncs;
    const double n = c[2];
    if (n <= 0) return 0.0;
    const int ix = L == 0 ? 0 : (L == 2 ? 1 : 4 + 2 * (L / 2 - 2));
    const int iw = L == 0 ? 2 : (L == 2 ? 3 : ix + 1);
    return (c[ix] - s3 * c[iw]) / n;
  };
  for (int o = wid; o < nmult * nn; o += nwarps) {
    const int e = o / nn, ij = o % nn, i = ij / nb, j = ij % nb;
    const double ni = cross_m[(size_t)i * ncs + 2], nj = cross_m[(size_t)j * ncs + 2];
    double s = 0.0;
    for (int c = 0; c < ncombo; ++c) s += coef[(size_t)e * ncombo + c] * red[(size_t)c * nn + ij];
    const double raw = (ni > 0 && nj > 0) ? s / (i33 * ni * nj * ncell) : 0.0;
    double sn = 0.0;
    if (shot == 2 && ni > 0 && nj > 0) {
      const double* d = desc + (size_t)e * SUGI_DESC;
      const int l1 = (int)d[0], l2 = (int)d[1];
      double t12 = 0.0;
      for (int c = 0; c < ncombo; ++c) t12 += coef[(size_t)e * ncombo + c] * red[(size_t)(ncombo + c) * nn + ij];
      // A or C (k = 0 or 2) of (l, m) on bin b, m of either sign
      auto get = [&](int l, int m, int b, int k, double& re, double& im) {
        const int am = m < 0 ? -m : m;
        const double* p = sbins + (size_t)b * NSB + 4 * (l * (l + 1) / 2 + am) + k;
        re = p[0];
        im = p[1];
        if (m < 0) {
          const int ph = am + (k == 2 ? l : 0);
          im = -im;
          if (ph & 1) {
            re = -re;
            im = -im;
          }
        }
      };
      double rest = 0.0;
      const int mm = l1 < l2 ? l1 : l2;
      for (int m = -mm; m <= mm; ++m) {
        double a1r, a1i, c1r, c1i, a2r, a2i, c2r, c2i;
        get(l1, m, i, 0, a1r, a1i);
        get(l1, m, i, 2, c1r, c1i);
        get(l2, -m, j, 0, a2r, a2i);
        get(l2, -m, j, 2, c2r, c2i);
        const double t = (a1r * c2r - a1i * c2i) + (c1r * a2r - c1i * a2i) - 2.0 * s3 * (a1r * a2r - a1i * a2i);
        rest += d[4 + m + 4] * t;
      }
      sn = (t12 / ncell + d[3] * rest) / (i33 * ni * nj);
    } else if (shot == 1 && ni > 0 && nj > 0) {
      const double* d = desc + (size_t)e * SUGI_DESC;
      const int l1 = (int)d[0], l2 = (int)d[1], L = (int)d[2];
      double v = 0.0;
      if (l1 == 0 && l2 == 0 && L == 0) v += s3;
      if (l1 == L && l2 == 0) v += (2 * L + 1) * shell(cross_m, L, i);
      if (l2 == L && l1 == 0) v += (2 * L + 1) * shell(cross_m, L, j);
      const double ci = kmin + (i + 0.5) * dk, cj = kmin + (j + 0.5) * dk;
      const double lo = fabs(ci - cj) + 0.5 * dk, hi = ci + cj - 0.5 * dk;
      const int nmin = l1 < l2 ? l1 : l2;
      double num = 0.0, den = 0.0;
      for (int m = lane; m < nq; m += 32) {
        const double cm = (m + 0.5) * dk;
        const double nm = cross_q[(size_t)m * ncs + 2];
        if (cm < lo - 1e-9 * dk || cm > hi + 1e-9 * dk || nm <= 0) continue;
        const double c13 = fmin(1.0, fmax(-1.0, (cj * cj - ci * ci - cm * cm) / (2.0 * ci * cm)));
        const double c23 = fmin(1.0, fmax(-1.0, (ci * ci - cj * cj - cm * cm) / (2.0 * cj * cm)));
        double q = 0.0;
        for (int n = -nmin; n <= nmin; ++n)
          q += ((n & 1) ? -1.0 : 1.0) * racah_assoc(l1, n, c13) * racah_assoc(l2, -n, c23) * d[4 + n + 4];
        num += nm / cm * q * shell(cross_q, L, m);
        den += nm / cm;
      }
      for (int off = 16; off > 0; off >>= 1) {   // fixed tree: the same sum on every lane
        num += __shfl_xor_sync(0xffffffffu, num, off);
        den += __shfl_xor_sync(0xffffffffu, den, off);
      }
      if (den > 0) v += d[3] * num / den;
      sn = v / i33;
    }
    if (lane == 0) {
      out[o] = raw - sn;
      out[(size_t)nmult * nn + o] = sn;
    }
  }
  if (blockIdx.x == 0) {
    for (int b = threadIdx.x; b < nb; b += blockDim.x) out[(size_t)2 * nmult * nn + b] = cross_m[(size_t)b * ncs + 2];
    if (threadIdx.x < 8) out[(size_t)2 * nmult * nn + nb + threadIdx.x] = sc[threadIdx.x];
  }
}

// Per-bin lattice sums of the TripoSH FFT-method shot noise, for l <= 4 and 0 <= m <= l at index
// 4 (l(l+1)/2 + m): Re A, Im A, Re C, Im C with A_l^m(b) = sum_{q in b} y_l^{m*}(qhat) and
// C_l^m(b) = sum_{q in b} y_l^{m*}(qhat) X(q) N^*(q), y in the line-of-sight frame.  A row kz > 0 of
// the half spectrum stands for q and -q: y^{m*}(-qhat) = (-1)^l y^{m*}(qhat), XN^*(-q) = conj XN^*(q).
template <typename T, int N>
__global__ void __launch_bounds__(BT)
k_sugi_binsums(const cplx<T>* __restrict__ X0, const cplx<T>* __restrict__ XN, int KY, const LosFrame fr,
               const int16_t* __restrict__ tab_m, int nbm, double* __restrict__ part) {
  constexpr int NW = BT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* pm = part + ((size_t)blockIdx.x * NW + warp) * nbm * NSB;
  const int nyr = 2 * KY + 1;
  const int nrows = (KY + 1) * nyr;
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int kz = r / nyr;
    const int jy = r % nyr - KY;
    const int ky = jy < 0 ? jy + N : jy;
    for (int jb = warp * 32; jb < N; jb += blockDim.x) {
      const int j = jb + lane;
      const int i = j < N / 2 ? j : j - N;
      const int n2 = i * i + jy * jy + kz * kz;
      int bm = -1;
      T vals[NSB];
#pragma unroll
      for (int q = 0; q < NSB; ++q) vals[q] = T(0);
      if (j < N && n2 > 0 && i != -N / 2 && jy != -N / 2) bm = tab_m[n2];
      if (bm >= 0) {
        const size_t idx = ((size_t)kz * N + ky) * N + j;
        const cplx<T> a = X0[idx], b = XN[idx];
        const T xr = a.x * b.x + a.y * b.y, xi = a.y * b.x - a.x * b.y;   // X N^*
        const T inv = T(1) / sqrt(T(n2));
        const T ii = T(i), jj = T(jy), zz = T(kz);
        const T ux = (ii * T(fr.e1[0]) + jj * T(fr.e1[1]) + zz * T(fr.e1[2])) * inv;
        const T uy = (ii * T(fr.e2[0]) + jj * T(fr.e2[1]) + zz * T(fr.e2[2])) * inv;
        const T uz = (ii * T(fr.e3[0]) + jj * T(fr.e3[1]) + zz * T(fr.e3[2])) * inv;
#pragma unroll
        for (int l = 0; l <= 4; ++l)
#pragma unroll
          for (int m = 0; m <= l; ++m) {
            T yr, yi;
            ylm_frame<T>(l, m, ux, uy, uz, yr, yi);
            const T sr = yr, si = -yi;   // y^{m*}
            const T mir = kz > 0 ? ((l & 1) ? T(-1) : T(1)) : T(0);
            const int o = 4 * (l * (l + 1) / 2 + m);
            vals[o] = sr * (T(1) + mir);
            vals[o + 1] = si * (T(1) + mir);
            // y* XN + mir y* conj(XN)
            vals[o + 2] = sr * xr - si * xi + mir * (sr * xr + si * xi);
            vals[o + 3] = sr * xi + si * xr + mir * (si * xr - sr * xi);
          }
      }
      seg_accumulate<T, NSB>(lane, bm, vals, pm);
    }
  }
}

// reduce per-warp cross partials into [bin][NCROSS] in a fixed order
// one warp per (bin, sum): strided lane sums then a fixed shuffle tree (reproducible order)
__global__ void k_cross_reduce(const double* __restrict__ part, int nrec, int nb, int ns, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x / 32;
  for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < nb * ns; e += gridDim.x * wpb) {
    double s = 0;
    for (int r = lane; r < nrec; r += 32) s += part[(size_t)r * nb * ns + e];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) out[e] = s;
  }
}

// Sum of per-CTA partials part[q][e] over q for every entry e.  A block takes 32 consecutive
// entries (one per lane, so every load of a warp is contiguous) and splits the CTAs q over its
// PR_SLICES warps (slice y sums q = y, y + PR_SLICES, ...); the slice sums are then added in slice
// order, so the result does not depend on scheduling.
constexpr int PR_SLICES = 16;
__global__ void __launch_bounds__(32 * PR_SLICES) k_part_reduce(const double* __restrict__ part, int nparts,
                                                                int64_t nent, double* __restrict__ out) {
  __shared__ double sl[PR_SLICES][33];
  const int lane = threadIdx.x & 31, y = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  double s = 0.0;
  if (e < nent) {
#pragma unroll 4
    for (int q = y; q < nparts; q += PR_SLICES) s += part[(size_t)q * nent + e];
  }
  sl[y][lane] = s;
  __syncthreads();
  if (y == 0 && e < nent) {
    double t = 0.0;
    for (int r = 0; r < PR_SLICES; ++r) t += sl[r][lane];
    out[e] = t;
  }
}

// reduce the indicator-triple partials over CTAs: nt[p][k]
// Sum_x I_i I_j I_k = ncell * (number of closed wavevector triples q_i + q_j + q_k = 0).  With every
// shell inside |q| <= k_N/2 no triple aliases across the grid, so the count is an exact integer and
// the sum is rounded to ncell * round(count): this removes the rounding error of the float shell
// fields from the normalisation whenever it is below half a triangle.
// (round_count = 0: the Legendre-weighted count sum_x L_2 I_i I_j I_k, not an integer, is kept as is)
__global__ void k_nt_reduce(const double* __restrict__ part, int nparts, int npair, int nslots, int nb,
                            double ncell, int round_count, double* __restrict__ nt) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < npair * nb; e += gridDim.x * blockDim.x) {
    const int p = e / nb, k = e % nb;
    double s = 0;
    for (int c = 0; c < nparts; ++c) s += part[((size_t)c * npair + p) * nslots + k];
    nt[e] = round_count ? rint(s / ncell) * ncell : s;
  }
}

// ------------------------------------------------------------------------------------------
// host helpers
// ------------------------------------------------------------------------------------------
// Wigner 3j symbol for integer arguments by the Racah formula (float64; the factorials stay exact
// for the arguments used here, j1 + j2 + j3 + 1 <= 17)
static double wigner3j_host(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0 || j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  auto fact = [](int n) {
    double f = 1.0;
    for (int q = 2; q <= n; ++q) f *= q;
    return f;
  };
  const double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
  const double pre =
      std::sqrt(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) * fact(j3 + m3) * fact(j3 - m3));
  const int tmin = std::max(0, std::max(j2 - j3 - m1, j1 - j3 + m2));
  const int tmax = std::min(j1 + j2 - j3, std::min(j1 - m1, j2 + m2));
  double sum = 0.0;
  for (int t = tmin; t <= tmax; ++t)
    sum += ((t & 1) ? -1.0 : 1.0) / (fact(t) * fact(j3 - j2 + t + m1) * fact(j3 - j1 + t - m2) *
                                     fact(j1 + j2 - j3 - t) * fact(j1 - t - m1) * fact(j2 - t + m2));
  const int ph = j1 - j2 - m3;
  return ((ph % 2) != 0 ? -1.0 : 1.0) * pre * sum;
}

struct Tri {
  std::vector<int> tri;   // [ntri][3]
  std::vector<int> pij;   // pair (i | j << 16), lexicographic i <= j
};

// centre closure rule c_k <= c_i + c_j, float64 with a relative slack of 1e-9 dk (the same
// expression as the test oracle; host code is compiled without floating-point contraction)
Tri make_triangles(const npc_kbins& kb) {
  Tri T;
  const int nb = kb.nbins;
  std::vector<double> c(nb);
  for (int b = 0; b < nb; ++b) c[b] = kb.kmin + (b + 0.5) * kb.dk;
  for (int i = 0; i < nb; ++i)
    for (int j = i; j < nb; ++j) {
      T.pij.push_back(i | (j << 16));
      for (int k = j; k < nb; ++k)
        if (c[k] <= c[i] + c[j] + 1e-9 * kb.dk) {
          T.tri.push_back(i);
          T.tri.push_back(j);
          T.tri.push_back(k);
        }
    }
  return T;
}

// the smallest compiled transform length >= need (and <= n; float64 up to 256)
int shell_grid_size(int need, int n, bool fp64) {
  static const int sizes[] = {16, 32, 48, 64, 96, 128, 192, 256, 512};
  for (int s : sizes) {
    if (s > n || (fp64 && s > 256)) break;
    if (s >= need) return s;
  }
  return n;
}

struct ShellLaunch {
  const void* X;
  const void* XN;   // N-field spectrum for src = 2 fields, or null
  const void* X2;   // Yamamoto X_2 for src = 3 fields, or null
  const void* X1;   // Yamamoto X_1, X_3 for src = 4, 5 fields, or null
  const void* X3;
  const void* XB;   // tracers 2 and 3 of a multi-tracer bispectrum (src = 6, 7), or null
  const void* XC;
  const void* XCOMP;  // component spectra for src = 8 fields (KZX n^2 each), or null
  int KZX, nfine;
  const ShellField* fields;
  int nfield, Kmax;
  const int16_t* tab;
  int n2cap;
  LosFrame frame;
  int has_yw;       // some field carries a TripoSH weight (mult 2)
  const int* plane_f;
  const int* plane_kz;
  int nplanes;
  const int *za, *zb, *oa, *ob;
  int nzp;
  unsigned* fmax;   // per R field: bits of the largest |value| written (float fields), or null
};

// the three shell passes on the NS grid
template <typename T, int NS>
npc_status shell_passes(npc_ctx* ctx, const ShellLaunch& sl, cplx<T>* T1, cplx<T>* T2, T* R) {
  using C = cplx<T>;
  const void* twp;
  NPC_TRY(get_twiddles(ctx, NS, sizeof(T) == 8 ? NPC_PREC_FP64 : NPC_PREC_MIXED, &twp));
  const C* tw = (const C*)twp;
  {
    const size_t smem = sizeof(C) * (8 * NS + (size_t)RowGroups<NS, BT>::NBUF * row_pad_len<NS>()) +
                        sizeof(T) * NS + sizeof(int) * 2 * NS;
    auto kern = sl.has_yw ? k_shell_x<T, NS, true> : k_shell_x<T, NS, false>;
    NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int nrows = (sl.Kmax + 1) * (2 * sl.Kmax + 1);
    kern<<<std::min(nrows, ctx->num_sms * 4), BT, smem, ctx->stream>>>(
        (const C*)sl.X, (const C*)sl.XN, (const C*)sl.X2, (const C*)sl.X1, (const C*)sl.X3, (const C*)sl.XB,
        (const C*)sl.XC, (const C*)sl.XCOMP, sl.KZX, sl.nfine,
        sl.fields, sl.nfield, sl.Kmax, sl.tab,
        sl.n2cap, sl.frame, tw, T1);
    NPC_LAUNCH(ctx);
  }
  constexpr int TX = BCol<NS>::TX;
  const size_t smem = sizeof(C) * (NS + (size_t)NS * TX);
  auto ky = k_shell_y<T, NS>;
  NPC_CUDA(ctx, cudaFuncSetAttribute(ky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int p0 = 0; p0 < sl.nplanes; p0 += 65535) {
    const int np_ = std::min(65535, sl.nplanes - p0);
    ky<<<dim3(NS / TX, np_), BCol<NS>::THREADS, smem, ctx->stream>>>(T1, sl.fields, sl.plane_f + p0,
                                                                     sl.plane_kz + p0, tw, T2);
    NPC_LAUNCH(ctx);
  }
  auto kz = k_shell_z<T, NS>;
  NPC_CUDA(ctx, cudaFuncSetAttribute(kz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kz<<<dim3(NS / TX, NS, sl.nzp), BCol<NS>::THREADS, smem, ctx->stream>>>(T2, sl.fields, sl.za, sl.zb, sl.oa, sl.ob,
                                                                          tw, R, sl.nfield, sl.fmax);
  NPC_LAUNCH(ctx);
  return NPC_OK;
}

template <typename T>
npc_status shell_dispatch(npc_ctx* ctx, int NS, const ShellLaunch& sl, cplx<T>* T1, cplx<T>* T2, T* R) {
  switch (NS) {
    case 16: return shell_passes<T, 16>(ctx, sl, T1, T2, R);
    case 32: return shell_passes<T, 32>(ctx, sl, T1, T2, R);
    case 48: return shell_passes<T, 48>(ctx, sl, T1, T2, R);
    case 64: return shell_passes<T, 64>(ctx, sl, T1, T2, R);
    case 96: return shell_passes<T, 96>(ctx, sl, T1, T2, R);
    case 128: return shell_passes<T, 128>(ctx, sl, T1, T2, R);
    case 192: return shell_passes<T, 192>(ctx, sl, T1, T2, R);
    case 256: return shell_passes<T, 256>(ctx, sl, T1, T2, R);
  }
  if constexpr (sizeof(T) == 4) {
    if (NS == 512) return shell_passes<T, 512>(ctx, sl, T1, T2, R);
  }
  return set_err(ctx, NPC_ERR_UNSUPPORTED, "shell grid %d not supported at this precision", NS);
}

template <typename T, int N>
npc_status bispec_impl(npc_ctx* ctx, const npc_mesh_spec& m, const npc_kbins& kb, int scoc_mask, int tripo_mask,
                       int shot, const DevCatalog& d, const DevCatalog* r, double* sc, double* dev_out,
                       int64_t out_len, const SugiReq* sug = nullptr, const CrossReq* crq = nullptr,
                       double* sc_own = nullptr) {
  // multi-tracer bispectra (crq): `sc` holds the combined normalisation, `sc_own` tracer 1's own
  // scalars (its FKP field needs its alpha)
  double* const sc_paint = (crq && sc_own) ? sc_own : sc;
  using C = cplx<T>;
  const double kf = 2.0 * M_PI / m.box;
  const double kmax = kb.kmin + kb.nbins * kb.dk;
  const int nb = kb.nbins;
  const int K = (int)std::ceil(kmax / kf) + 1;            // shells
  const int K2 = std::min((int)std::ceil(2.0 * kmax / kf) + 2, N / 2 - 1);  // G fields, k3 shells
  const int nq = (int)std::ceil(2.0 * kmax / kb.dk) + 1;
  const int n2cap = (int)std::floor(std::pow(2.0 * kmax / kf, 2)) + 1;
  const int KZ = K2 + 1;
  const int nphase = m.interlace ? 2 : 1;
  const Geom geo = [&] {
    Geom g{};
    g.n = N;
    g.h = m.box / N;
    for (int a = 0; a < 3; ++a) g.o[a] = m.origin[a];
    g.global_los = 1;
    return g;
  }();
  // global line of sight (only the l = 2 terms use it; the monopoles of a survey need none)
  double l3[3] = {0.0, 0.0, 1.0};
  if (m.los == 1) {
    const double ll = std::sqrt(m.los_dir[0] * m.los_dir[0] + m.los_dir[1] * m.los_dir[1] + m.los_dir[2] * m.los_dir[2]);
    for (int a = 0; a < 3; ++a) l3[a] = m.los_dir[a] / ll;
  }
  // frame of the TripoSH weights: e3 the line of sight, e1 from x (or y when the line of sight is
  // close to x) with its e3 component removed, e2 = e3 x e1 (x, y, z themselves for a line of sight
  // along z)
  LosFrame frame{};
  {
    double a[3] = {std::fabs(l3[0]) < 0.9 ? 1.0 : 0.0, std::fabs(l3[0]) < 0.9 ? 0.0 : 1.0, 0.0};
    const double ad = a[0] * l3[0] + a[1] * l3[1];
    double e1[3] = {a[0] - ad * l3[0], a[1] - ad * l3[1], a[2] - ad * l3[2]};
    const double n1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int q = 0; q < 3; ++q) {
      frame.e1[q] = e1[q] / n1;
      frame.e3[q] = l3[q];
    }
    frame.e2[0] = l3[1] * frame.e1[2] - l3[2] * frame.e1[1];
    frame.e2[1] = l3[2] * frame.e1[0] - l3[0] * frame.e1[2];
    frame.e2[2] = l3[0] * frame.e1[1] - l3[1] * frame.e1[0];
  }
  const bool sugi = sug != nullptr;
  // TripoSH with the line of sight to each grid point: G_L^M from y_L^M-weighted transforms and the
  // full m1 + m2 + M = 0 sum in the catalogue frame (raw estimates)
  const bool sugi_ep = sugi && m.los != 1 && !m.periodic;
  int sugi_lmask = 0;   // L > 0 of the requested TripoSH multipoles
  if (sugi_ep)
    for (int e = 0; e < sug->nmult; ++e)
      if (sug->L[e] > 0) sugi_lmask |= 1 << sug->L[e];
  // survey geometry with the line of sight to each grid point and an l = 2 request: Yamamoto X_2
  // from the Y_2m-weighted transforms instead of L_2(khat . los) X_0
  const bool yam = !m.periodic && m.los != 1 && (((scoc_mask | tripo_mask) & 4) != 0);
  // odd Scoccimarro multipoles l = 1, 3 (Sec. 2.1: the imaginary part of the closure sum), l on
  // leg 1: with the line of sight to each grid point the Yamamoto X_l of the Y_lm-weighted
  // transforms (yamo), otherwise L_l(qhat . los) X_0; raw estimates (no shot noise)
  const bool want1 = (scoc_mask & 2) != 0, want3 = (scoc_mask & 8) != 0;
  const bool yamo = !m.periodic && m.los != 1 && (want1 || want3);

  // 1. paint + forward transforms of F and N fields
  const size_t rs = sizeof(T);
  const size_t ncell = (size_t)N * N * N;
  void *ma, *mb = nullptr, *half;
  NPC_TRY(ws_get(ctx, "mesh.a", rs * ncell, &ma));
  if (nphase == 2) NPC_TRY(ws_get(ctx, "mesh.b", rs * ncell, &mb));
  PowerPlan plan{};
  plan.n = N;
  plan.nphase = nphase;
  plan.global_los = yam ? 0 : 1;
  plan.assign = m.assign;
  plan.kz_keep = KZ;
  plan.fl.nf = 0;
  // survey layout: component c = (l, m, part) with its phase-a and phase-b fields adjacent
  auto build_survey = [&](PowerPlan& pl, YamComps& yc, int lmask) {
    pl.fl.nf = 0;
    yc = YamComps{};
    auto comp = [&](int l, int mm, int part) {
      const int c = yc.nc++;
      yc.l[c] = (int8_t)l; yc.m[c] = (int8_t)mm; yc.part[c] = (int8_t)part;
      for (int ph = 0; ph < nphase; ++ph) {
        (ph == 0 ? yc.ia[c] : yc.ib[c]) = (int8_t)pl.fl.nf;
        Comp f;
        f.phase = (int8_t)ph; f.ell = (int8_t)l; f.m = (int8_t)mm; f.part = (int8_t)part;
        pl.fl.f[pl.fl.nf++] = f;
      }
    };
    comp(0, 0, PART_ONE);
    for (int l = 1; l <= 4; ++l) {
      if (!(lmask & (1 << l))) continue;
      comp(l, 0, PART_RE);
      for (int mm = 1; mm <= l; ++mm) {
        comp(l, mm, PART_RE);
        comp(l, mm, PART_IM);
      }
    }
    yc.nf = pl.fl.nf;
  };
  auto build_plain = [&](PowerPlan& pl) {
    pl.fl.nf = 0;
    for (int ph = 0; ph < nphase; ++ph) {
      Comp c;
      c.phase = (int8_t)ph; c.ell = 0; c.m = 0; c.part = PART_ONE;
      pl.fl.f[pl.fl.nf++] = c;
    }
  };
  YamComps ycF{}, ycN{};
  PowerPlan planN = plan;
  if (sugi_ep) build_survey(plan, ycF, sugi_lmask);
  else if (yam || yamo) build_survey(plan, ycF, ((yamo && want1) ? 2 : 0) | (yam ? 4 : 0) | ((yamo && want3) ? 8 : 0));
  else build_plain(plan);
  if (yam) build_survey(planN, ycN, 4);
  else build_plain(planN);
  plan.global_los = (yam || yamo || sugi_ep) ? 0 : 1;
  planN.global_los = yam ? 0 : 1;
  const Geom gyam = make_geom(m);   // observer-relative grid points for the Y weighting
  const Geom& gfwd = (yam || yamo || sugi_ep) ? gyam : geo;
  const Geom& gfwdN = yam ? gyam : geo;
  const int prec = sizeof(T) == 8 ? NPC_PREC_FP64 : NPC_PREC_MIXED;
  const size_t halfbytes = sizeof(C) * (size_t)plan.fl.nf * KZ * N * N;
  NPC_TRY(ws_get(ctx, "half", 2 * halfbytes, &half));
  C* halfF = (C*)half;
  C* halfN = (C*)((char*)half + halfbytes);
  NPC_TRY(stage_mark(ctx, "alloc"));
  NPC_TRY(launch_paint(ctx, d, r, m, 1, prec, sc_paint, ma, mb));
  NPC_TRY(stage_mark(ctx, "paint_fold"));
  NPC_TRY(run_forward_transforms(ctx, prec, plan, gfwd, ma, mb, halfF));
  if (shot) {
    NPC_TRY(launch_paint(ctx, d, r, m, 2, prec, sc, ma, mb));
    NPC_TRY(run_forward_transforms(ctx, prec, planN, gfwdN, ma, mb, halfN));
  }
  NPC_TRY(stage_mark(ctx, "forward_yz"));

  const void* twf;
  NPC_TRY(get_twiddles(ctx, N, prec, &twf));
  const C* tw = (const C*)twf;
  // 2. x pass + combine into X0 (and XN); survey l = 2 also X2 (and N2) at X + 2 xfs (+ 3 xfs), survey
  //    odd l the Yamamoto X1 at X + 4 xfs and X3 at X + 5 xfs
  C* X;
  const int nout = shot ? 2 : 1;
  const size_t xfs = (size_t)KZ * N * N;
  NPC_TRY(ws_get(ctx, "bis.X",
                 sizeof(C) * xfs * (sugi_ep ? ycF.nc : (crq ? 3 : (yamo ? 6 : (yam ? 4 : nout)))), (void**)&X));
  {
    const int nrows = KZ * (2 * K2 + 1);
    const int grid = std::min(nrows, ctx->num_sms * 4);
    auto assemble = [&](const C* src, const YamComps& yc, C* x0, C* x1, C* x2, C* x3, C* comps = nullptr) -> npc_status {
      const size_t smem = sizeof(C) * (2 * N + (size_t)(yc.nf + RowGroups<N, BT>::NBUF) * row_pad_len<N>()) +
                          sizeof(T) * (N / 2 + 2);
      if (smem > 227 * 1024) return set_err(ctx, NPC_ERR_UNSUPPORTED, "survey multipoles: mesh too large at this precision");
      auto kern = k_fft_x_assemble_yam<T, N>;
      NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<grid, BT, smem, ctx->stream>>>(src, nphase, KZ, K2, m.assign, ylm_norm_table(), yc, tw, x0, x1, x2, x3,
                                            comps);
      NPC_LAUNCH(ctx);
      return NPC_OK;
    };
    auto combine = [&](const C* src, C* dst) -> npc_status {
      const size_t smem =
          sizeof(C) * (2 * N + (size_t)(nphase + RowGroups<N, BT>::NBUF) * row_pad_len<N>()) + sizeof(T) * (N / 2 + 2);
      auto kern = k_fft_x_combine<T, N>;
      NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<grid, BT, smem, ctx->stream>>>(src, 1, nphase, KZ, K2, m.assign, tw, dst);
      NPC_LAUNCH(ctx);
      return NPC_OK;
    };
    if (sugi_ep)   // component c at X + c xfs; component 0 (the plain field) is X_0
      NPC_TRY(assemble(halfF, ycF, X, nullptr, nullptr, nullptr, X));
    else if (yam || yamo)
      NPC_TRY(assemble(halfF, ycF, X, (yamo && want1) ? X + 4 * xfs : nullptr, yam ? X + 2 * xfs : nullptr,
                       (yamo && want3) ? X + 5 * xfs : nullptr));
    else
      NPC_TRY(combine(halfF, X));
    if (shot) {
      if (yam) NPC_TRY(assemble(halfN, ycN, X + xfs, nullptr, X + 3 * xfs, nullptr));
      else NPC_TRY(combine(halfN, X + xfs));
    }
    // tracers 2 and 3 of a multi-tracer bispectrum: X at X + xfs and X + 2 xfs
    for (int t = 0; crq && t < 2; ++t) {
      NPC_TRY(launch_paint(ctx, crq->d[t], crq->has_r ? &crq->r[t] : nullptr, m, 1, prec, crq->sc[t], ma, mb));
      NPC_TRY(run_forward_transforms(ctx, prec, plan, gfwd, ma, mb, halfF));
      NPC_TRY(combine(halfF, X + (size_t)(1 + t) * xfs));
    }
  }
  NPC_TRY(stage_mark(ctx, "forward_x_combine"));

  // 3. shell sums for the shot noise
  const int16_t *tab_m, *tab_q;
  NPC_TRY(get_bin_table(ctx, N, m.box, kb, &tab_m, 2));
  npc_kbins qb{0.0, kb.dk, nq};
  NPC_TRY(get_bin_table(ctx, N, m.box, qb, &tab_q, 3));
  const int nsum_c = yam ? NCS : (sugi ? NCROSS_S : NCROSS);   // shell sums per bin
  double *cross_m, *cross_q, *mom = nullptr;
  NPC_TRY(ws_get(ctx, "bis.cross", sizeof(double) * nsum_c * (nb + nq) + sizeof(double) * 8, (void**)&cross_m));
  cross_q = cross_m + (size_t)nsum_c * nb;
  if (yam) mom = cross_q + (size_t)nsum_c * nq;
  {
    const int nrows = (K2 + 1) * (2 * K2 + 1);
    const int grid = std::min(nrows, ctx->num_sms * 2);
    const int nw = BT / 32;
    double* part;
    const size_t np = (size_t)grid * nw;
    NPC_TRY(ws_get(ctx, "bis.crosspart", sizeof(double) * np * nsum_c * (nb + nq), (void**)&part));
    NPC_CUDA(ctx, cudaMemsetAsync(part, 0, sizeof(double) * np * nsum_c * (nb + nq), ctx->stream));
    const C* XN = shot ? X + xfs : X;
    if (yam) {
      const C* N2 = shot ? X + 3 * xfs : X + 2 * xfs;
      k_bin_cross_survey<T, N><<<grid, BT, 0, ctx->stream>>>(X, X + 2 * xfs, XN, N2, K2, ylm_norm_table(), tab_m, nb,
                                                            tab_q, nq, n2cap, part, part + np * NCS * nb);
    } else if (sugi) {
      k_bin_cross<T, N, NCROSS_S><<<grid, BT, 0, ctx->stream>>>(X, XN, KZ, K2, l3[0], l3[1], l3[2], tab_m, nb, tab_q,
                                                               nq, n2cap, part, part + np * NCROSS_S * nb);
    } else {
      k_bin_cross<T, N><<<grid, BT, 0, ctx->stream>>>(X, XN, KZ, K2, l3[0], l3[1], l3[2], tab_m, nb, tab_q, nq, n2cap,
                                                     part, part + np * NCROSS * nb);
    }
    NPC_LAUNCH(ctx);
    k_cross_reduce<<<(nb * nsum_c + 3) / 4, 128, 0, ctx->stream>>>(part, (int)np, nb, nsum_c, cross_m);
    NPC_LAUNCH(ctx);
    k_cross_reduce<<<(nq * nsum_c + 3) / 4, 128, 0, ctx->stream>>>(part + np * nsum_c * nb, (int)np, nq, nsum_c,
                                                                 cross_q);
    NPC_LAUNCH(ctx);
    if (yam && shot) {
      // catalogue moments C_2m of the self term (data, then randoms scaled by -alpha^3)
      double* pm;
      NPC_TRY(ws_get(ctx, "bis.ympart", sizeof(double) * 5 * YM_BLOCKS * 2, (void**)&pm));
      const YNorm nrm = ylm_norm_table();
      auto moments = [&](const DevCatalog& c, double* out) {
        if (c.dtype == 1)
          k_cat_ylm2<double><<<YM_BLOCKS, YM_THREADS, 0, ctx->stream>>>(
              (const double*)c.pos, (const double*)c.w, c.n, m.observer[0], m.observer[1], m.observer[2], nrm, out);
        else
          k_cat_ylm2<float><<<YM_BLOCKS, YM_THREADS, 0, ctx->stream>>>(
              (const float*)c.pos, (const float*)c.w, c.n, m.observer[0], m.observer[1], m.observer[2], nrm, out);
      };
      moments(d, pm);
      NPC_LAUNCH(ctx);
      if (r) {
        moments(*r, pm + 5 * YM_BLOCKS);
        NPC_LAUNCH(ctx);
      }
      k_cat_ylm2_final<<<1, 32, 0, ctx->stream>>>(pm, pm + 5 * YM_BLOCKS, YM_BLOCKS, r ? 1 : 0, sc, mom);
      NPC_LAUNCH(ctx);
    }
  }
  NPC_TRY(stage_mark(ctx, "shot_shells"));

  // 4. shell fields
  const bool want2 = (scoc_mask & 4) != 0;
  const bool wantG0 = (tripo_mask & 1) != 0 || sugi, wantG2 = (tripo_mask & 4) != 0;
  // grid of the shell fields and triple products: shells reach |q_i| <= K and the full fields
  // |q_i| <= K2, so a closed triple sums to at most 3K (2K + K2 with the compressed estimator) per
  // axis; any grid of more points has no aliasing and gives the same sums up to (n/NS)^3, which
  // cancels in every normalised result (cell counts are those of the NS grid)
  // exact radii: shell modes (|q| < k_max) have integer components <= Ks, full-field modes
  // (|q|^2 <= n2cap) components <= KG
  const int Ks = std::max(1, (int)std::floor(kmax / kf));
  const int KG = std::max(1, std::min((int)std::floor(std::sqrt((double)n2cap)), N / 2 - 1));  // no Nyquist
  const int Kshell = (wantG0 || wantG2) ? std::max(Ks, KG) : Ks;
  const int need_ns = std::max((wantG0 || wantG2) ? 2 * Ks + KG + 1 : 3 * Ks + 1, 2 * Kshell + 1);
  const int NS = shell_grid_size(need_ns, N, sizeof(T) == 8);
  const size_t ncs = (size_t)NS * NS * NS;
  // triangle-count cache keyed by geometry and bins
  std::vector<char> ntkey(sizeof(int) + 3 * sizeof(double));
  {
    int n_ = N;
    double a[3] = {m.box, kb.kmin, kb.dk};
    std::memcpy(ntkey.data(), &n_, sizeof(int));
    std::memcpy(ntkey.data() + sizeof(int), a, 3 * sizeof(double));
    ntkey.push_back((char)nb);
    ntkey.push_back((char)sizeof(T));   // float and float64 shell fields give different rounding
    const char* nsb = reinterpret_cast<const char*>(&NS);
    ntkey.insert(ntkey.end(), nsb, nsb + sizeof(int));
  }
  const Tri tr = make_triangles(kb);
  const int ntri = (int)tr.tri.size() / 3, npair = (int)tr.pij.size();
  double* nt_sums = nullptr;
  const std::string ntname = slot_name(ctx, "bis.ntsums");
  if (!sugi) NPC_TRY(ws_get(ctx, ntname.c_str(), sizeof(double) * npair * nb, (void**)&nt_sums));
  auto it = ctx->host_cache_keys.find(ntname);
  const bool need_nt = !sugi && (it == ctx->host_cache_keys.end() || it->second != ntkey);

  // FFT-method shot noise: the l = 2 triplet count sum_x L_2 I_i I_j I_k is cached like N_T
  const bool fftshot = shot == 2;
  const bool want_nt2 = fftshot && want2;
  double* nt2_sums = nullptr;
  std::vector<char> nt2key = ntkey;
  nt2key.push_back('2');
  const std::string nt2name = slot_name(ctx, "bis.nt2sums");
  bool need_nt2 = false;
  if (want_nt2) {
    NPC_TRY(ws_get(ctx, nt2name.c_str(), sizeof(double) * npair * nb, (void**)&nt2_sums));
    auto it2 = ctx->host_cache_keys.find(nt2name);
    need_nt2 = it2 == ctx->host_cache_keys.end() || it2->second != nt2key;
  }

  std::vector<ShellField> fl;
  std::vector<int> ffam;   // field family (z-pass pairs stay within a family)
  auto add = [&](int src, int mult, int bin, int Kf, int fam, int lmult = 2) {
    ShellField f{};
    f.src = (int8_t)src; f.mult = (int8_t)mult; f.bin = (int16_t)bin; f.K = Kf;
    if (mult == 1) f.yl = (int8_t)lmult;   // L_l(mu) weight
    fl.push_back(f);
    ffam.push_back(fam);
  };
  for (int b = 0; b < nb; ++b) add(0, 0, b, Ks, 0);              // F0_b: R index b
  if (want2) for (int b = 0; b < nb; ++b) add(yam ? 3 : 0, yam ? 0 : 1, b, Ks, 1);   // F2_b: R index nb + b
  const int iF2 = want2 ? nb : -1;
  int iFB = 0, iFC = 0;   // shells of the legs 2 and 3 (F_0 of the same catalogue unless multi-tracer)
  if (crq) {
    iFB = (int)fl.size();
    for (int b = 0; b < nb; ++b) add(6, 0, b, Ks, 20);
    iFC = (int)fl.size();
    for (int b = 0; b < nb; ++b) add(7, 0, b, Ks, 21);
  }
  // odd multipoles: shells of -i X_l (survey: Yamamoto X_1 / X_3; global: L_l(mu) X_0)
  int iFodd[4] = {-1, -1, -1, -1};
  for (int l = 1; l <= 3; l += 2) {
    if (!(scoc_mask & (1 << l))) continue;
    iFodd[l] = (int)fl.size();
    for (int b = 0; b < nb; ++b) {
      if (yamo) add(l == 1 ? 4 : 5, 0, b, Ks, 10 + l);
      else add(0, 1, b, Ks, 10 + l, l);
    }
  }
  const int iI = (int)fl.size();
  if (need_nt || fftshot) for (int b = 0; b < nb; ++b) add(1, 0, b, Ks, 2);   // I_b
  const int iG = (int)fl.size();
  int ng = 0;
  const int gsrc = crq ? 7 : 0;   // the compressed estimator's full-range field: leg 3's tracer
  if (wantG0) { add(gsrc, 0, -1, KG, 3); ng++; }
  if (wantG2) { add(yam ? 3 : gsrc, yam ? 0 : 1, -1, KG, 3); ng++; }
  int iS0 = -1, iS2 = -1, iI2 = -1, iSF = -1, iLF = -1;
  int ntl = 0, tls[2] = {0, 0};   // compressed multipoles requested
  for (int l = 0; l <= 2; l += 2)
    if (tripo_mask & (1 << l)) tls[ntl++] = l;
  if (fftshot && !sugi) {
    iS0 = (int)fl.size();
    for (int b = 0; b < nb; ++b) add(2, 0, b, Ks, 4);            // sum_{q in b} X_0 N_0^* e^{iqx}
    if (want2) {
      iS2 = (int)fl.size();
      for (int b = 0; b < nb; ++b) add(2, 1, b, Ks, 5);          // the same with L_2(mu)
      iI2 = (int)fl.size();
      for (int b = 0; b < nb; ++b) add(1, 1, b, Ks, 6);          // L_2(mu) indicators
    }
    if (ntl > 0) {   // compressed estimator: full-range fields of L_l X_0 N_0^* and of L_l
      iSF = (int)fl.size();
      for (int e = 0; e < ntl; ++e) add(2, tls[e] == 2 ? 1 : 0, -1, KG, 7);
      iLF = (int)fl.size();
      for (int e = 0; e < ntl; ++e) add(1, tls[e] == 2 ? 1 : 0, -1, KG, 8);
    }
  }
  // TripoSH shell fields: the parts of F_l^m(x; k_b), 0 <= m <= min(l1, l2), of every l requested
  // (F_0^0 is F0_b above); sfield[l][m][part] = R index of bin 0, or -1
  int sfield[5][5][2], ifield[5][5][2], iXN = -1;   // ifield: the indicator versions (FFT-method shot noise)
  for (int l = 0; l < 5; ++l)
    for (int mm = 0; mm < 5; ++mm) sfield[l][mm][0] = sfield[l][mm][1] = ifield[l][mm][0] = ifield[l][mm][1] = -1;
  // endpoint TripoSH: the real triple products of the full sub-configuration sum.  With
  // F_l^{-m} = (-1)^{l+m} F_l^{m*}, G_L^{-M} = (-1)^M G_L^{M*} (both from the reality of F(x)) and
  // G_L^M = c_L (G[Re] - i G[Im]), c_L = sqrt(4 pi/(2L+1)) (G[Re], G[Im] the fields of the transforms
  // of F Re Y_LM and F Im Y_LM), every (m1, m2, M = -m1-m2) term is a product of the parts (real,
  // imaginary) of the |m| fields, and Re(z1 z2 z3) = x1 x2 x3 - x1 y2 y3 - y1 x2 y3 - y1 y2 x3.
  // For l1 + l2 odd (odd L) the sum is imaginary and its imaginary part is reported (the rule of
  // Sec. 2.1 for odd multipoles): Im(z1 z2 z3) = x1 x2 y3 + x1 y2 x3 + y1 x2 x3 - y1 y2 y3.
  struct EpKey {
    int l1, a1, p1, l2, a2, p2, L, A3, p3;
  };
  std::vector<EpKey> ep_keys;
  std::vector<std::vector<std::pair<int, double>>> ep_terms;
  int gfield[5][5][2];
  for (int l = 0; l < 5; ++l)
    for (int mm = 0; mm < 5; ++mm) gfield[l][mm][0] = gfield[l][mm][1] = -1;
  if (sugi_ep) {
    ep_terms.resize(sug->nmult);
    auto key_of = [&](const EpKey& k) {
      for (size_t q = 0; q < ep_keys.size(); ++q) {
        const EpKey& o = ep_keys[q];
        if (o.l1 == k.l1 && o.a1 == k.a1 && o.p1 == k.p1 && o.l2 == k.l2 && o.a2 == k.a2 && o.p2 == k.p2 &&
            o.L == k.L && o.A3 == k.A3 && o.p3 == k.p3)
          return (int)q;
      }
      ep_keys.push_back(k);
      return (int)ep_keys.size() - 1;
    };
    for (int e = 0; e < sug->nmult; ++e) {
      const int l1 = sug->l1[e], l2 = sug->l2[e], L = sug->L[e];
      const double hN = wigner3j_host(l1, l2, L, 0, 0, 0) * (2 * l1 + 1) * (2 * l2 + 1) * (2 * L + 1);
      const double cL = L == 0 ? 1.0 : std::sqrt(4.0 * M_PI / (2 * L + 1));
      for (int m1 = -l1; m1 <= l1; ++m1)
        for (int m2 = -l2; m2 <= l2; ++m2) {
          const int M = -m1 - m2;
          if (std::abs(M) > L) continue;
          const double w = wigner3j_host(l1, l2, L, m1, m2, M);
          if (w == 0.0) continue;
          const int a1 = std::abs(m1), a2 = std::abs(m2), A3 = std::abs(M);
          const double s1 = (m1 < 0 && ((l1 + a1) & 1)) ? -1.0 : 1.0, t1 = m1 < 0 ? -1.0 : 1.0;
          const double s2 = (m2 < 0 && ((l2 + a2) & 1)) ? -1.0 : 1.0, t2 = m2 < 0 ? -1.0 : 1.0;
          const double s3 = (M < 0 && (A3 & 1)) ? -1.0 : 1.0, t3 = M < 0 ? -1.0 : 1.0;
          const double base = hN * w * s1 * s2 * s3;
          const bool imag = ((l1 + l2) & 1) != 0;
          const int pr[4][3] = {{0, 0, 0}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};
          const int pi[4][3] = {{0, 0, 1}, {0, 1, 0}, {1, 0, 0}, {1, 1, 1}};
          const double sgr[4] = {1.0, -t2 * t3, -t1 * t3, -t1 * t2};
          const double sgi[4] = {t3, t2, t1, -t1 * t2 * t3};
          const int (&pp)[4][3] = imag ? pi : pr;
          const double* sg = imag ? sgi : sgr;
          for (int q = 0; q < 4; ++q) {
            const int p1 = pp[q][0], p2 = pp[q][1], p3 = pp[q][2];
            if (a1 == 0 && p1 == ((l1 & 1) ? 0 : 1)) continue;   // vanishing part of an m = 0 shell
            if (a2 == 0 && p2 == ((l2 & 1) ? 0 : 1)) continue;
            if (A3 == 0 && p3 == 1) continue;                    // G_L^0 is real
            const double gscale = p3 == 0 ? cL : -cL;
            ep_terms[e].push_back({key_of(EpKey{l1, a1, p1, l2, a2, p2, L, A3, p3}), base * sg[q] * gscale});
          }
        }
    }
    // shells F_l^m parts (catalogue frame) and the G_L^M parts (full range, from the components)
    sfield[0][0][0] = 0;
    int fam = 20;
    auto need_shell = [&](int l, int a, int p) {
      if (sfield[l][a][p] >= 0) return;
      sfield[l][a][p] = (int)fl.size();
      for (int b = 0; b < nb; ++b) {
        add(0, 2, b, Ks, fam);
        fl.back().yl = (int8_t)l;
        fl.back().ym = (int8_t)a;
        fl.back().ypart = (int8_t)p;
      }
      ++fam;
    };
    for (const EpKey& k : ep_keys) {
      need_shell(k.l1, k.a1, k.p1);
      need_shell(k.l2, k.a2, k.p2);
      if (k.L == 0) {
        gfield[0][0][0] = iG;
        continue;
      }
      if (gfield[k.L][k.A3][k.p3] >= 0) continue;
      int comp = -1;
      for (int c = 0; c < ycF.nc; ++c)
        if (ycF.l[c] == k.L && ycF.m[c] == k.A3 && ycF.part[c] == (k.p3 ? PART_IM : PART_RE)) comp = c;
      if (comp < 0) return set_err(ctx, NPC_ERR_INVALID_ARG, "TripoSH: missing y_L^M component");
      gfield[k.L][k.A3][k.p3] = (int)fl.size();
      add(8, 0, -1, KG, fam++);
      fl.back().comp = (int8_t)comp;
    }
  } else if (sugi) {
    sfield[0][0][0] = 0;
    int fam = 20;
    for (int e = 0; e < sug->nmult; ++e) {
      const int l1 = sug->l1[e], l2 = sug->l2[e], mmax = std::min(l1, l2);
      for (int side = 0; side < 2; ++side) {
        const int l = side ? l2 : l1;
        for (int mm = 0; mm <= mmax; ++mm)
          for (int part = 0; part < 2; ++part) {
            // m = 0: the imaginary part of an even-l field and the real part of an odd-l one vanish
            if (mm == 0 && part == ((l & 1) ? 0 : 1)) continue;
            if (sfield[l][mm][part] >= 0) continue;
            sfield[l][mm][part] = (int)fl.size();
            for (int b = 0; b < nb; ++b) {
              add(0, 2, b, Ks, fam);
              fl.back().yl = (int8_t)l;
              fl.back().ym = (int8_t)mm;
              fl.back().ypart = (int8_t)part;
            }
            ++fam;
          }
      }
    }
    if (fftshot) {
      // FFT-method shot noise: the same parts of the y-weighted indicator shells, and the
      // full-range field of X N^*
      ifield[0][0][0] = iI;
      for (int l = 0; l < 5; ++l)
        for (int mm = 0; mm < 5; ++mm)
          for (int part = 0; part < 2; ++part) {
            if (sfield[l][mm][part] < 0 || (l == 0 && mm == 0)) continue;
            ifield[l][mm][part] = (int)fl.size();
            for (int b = 0; b < nb; ++b) {
              add(1, 2, b, Ks, fam);
              fl.back().yl = (int8_t)l;
              fl.back().ym = (int8_t)mm;
              fl.back().ypart = (int8_t)part;
            }
            ++fam;
          }
      iXN = (int)fl.size();
      add(2, 0, -1, KG, fam++);
    }
  }
  const int nfield = (int)fl.size();
  int64_t o1 = 0, o2 = 0;
  std::vector<int> plane_f, plane_kz;
  for (int f = 0; f < nfield; ++f) {
    fl[f].off1 = o1;
    fl[f].off2 = o2;
    o1 += (int64_t)(fl[f].K + 1) * (2 * fl[f].K + 1) * NS;
    o2 += (int64_t)(fl[f].K + 1) * NS * NS;
    for (int kz = 0; kz <= fl[f].K; ++kz) {
      plane_f.push_back(f);
      plane_kz.push_back(kz);
    }
  }
  // pairs for the z pass: consecutive fields of the same family (F0, F2, I, G) and the same K, so
  // that the rounding of every field (a pair shares one complex transform) does not depend on
  // whether the cached indicator fields are recomputed in this call
  auto family = [&](int f) { return ffam[f]; };
  std::vector<int> za, zb;
  for (int f = 0; f < nfield;) {
    if (f + 1 < nfield && fl[f + 1].K == fl[f].K && family(f + 1) == family(f)) {
      za.push_back(f);
      zb.push_back(f + 1);
      f += 2;
    } else {
      za.push_back(f);
      zb.push_back(-1);
      f += 1;
    }
  }
  const int nzp = (int)za.size();
  // device tables (one upload per call; small)
  std::vector<char> tables;
  auto push_bytes = [&](const void* p, size_t n) {
    const size_t o = tables.size();
    tables.resize(o + ((n + 15) / 16) * 16);
    std::memcpy(tables.data() + o, p, n);
    return o;
  };
  const size_t t_fields = push_bytes(fl.data(), sizeof(ShellField) * nfield);
  const size_t t_pf = push_bytes(plane_f.data(), sizeof(int) * plane_f.size());
  const size_t t_pk = push_bytes(plane_kz.data(), sizeof(int) * plane_kz.size());
  const size_t t_za = push_bytes(za.data(), sizeof(int) * nzp);
  const size_t t_zb = push_bytes(zb.data(), sizeof(int) * nzp);
  const size_t t_oa = push_bytes(za.data(), sizeof(int) * nzp);  // R index = field index
  const size_t t_ob = push_bytes(zb.data(), sizeof(int) * nzp);
  const size_t t_tri = push_bytes(tr.tri.data(), sizeof(int) * tr.tri.size());
  const size_t t_pij = push_bytes(tr.pij.data(), sizeof(int) * tr.pij.size());
  // triple-product row order: pairs sorted by (j, i)
  std::vector<int> row_pair(tr.pij.size());
  for (size_t q = 0; q < row_pair.size(); ++q) row_pair[q] = (int)q;
  std::stable_sort(row_pair.begin(), row_pair.end(), [&](int a, int b) {
    const int ja = tr.pij[a] >> 16, jb = tr.pij[b] >> 16;
    return ja != jb ? ja < jb : (tr.pij[a] & 0xffff) < (tr.pij[b] & 0xffff);
  });
  const size_t t_rowp = push_bytes(row_pair.data(), sizeof(int) * row_pair.size());
  // TripoSH: combinations (l1, l2, m >= 0, part) and their weight in each multipole.  With
  // F_l^{-m} = (-1)^{l+m} F_l^{m*} (Eq. sugi_F_and_G), G_L^M = delta_M0 G in the line-of-sight frame
  // and (l1 l2 L; -m m 0) = (l1 l2 L; m -m 0) for even l1 + l2 + L, the m and -m sub-configurations
  // both contribute (-1)^{l2+m} (l1 l2 L; m -m 0) sum_x (Re F1 Re F2 + Im F1 Im F2) G: real part of
  // the product (Eq. sym_sugi).
  struct SCombo {
    int l1, l2, m, part;
    int fa = -1, fg = -1, fc = -1;   // endpoint TripoSH: the R indices of the three operands
  };
  std::vector<SCombo> combos;
  std::vector<double> scoef;
  size_t t_spij = 0, t_srow = 0, t_scoef = 0, t_sdesc = 0;
  if (sugi_ep) {
    for (const EpKey& k : ep_keys) {
      SCombo cb{k.l1, k.l2, k.a1, k.p1};
      cb.fa = sfield[k.l1][k.a1][k.p1];
      cb.fg = gfield[k.L][k.A3][k.p3];
      cb.fc = sfield[k.l2][k.a2][k.p2];
      combos.push_back(cb);
    }
    scoef.assign((size_t)sug->nmult * combos.size(), 0.0);
    for (int e = 0; e < sug->nmult; ++e)
      for (const auto& tw : ep_terms[e]) scoef[(size_t)e * combos.size() + tw.first] += tw.second;
  }
  if (sugi) {
    auto combo_of = [&](int l1, int l2, int mm, int part) {
      for (size_t c = 0; c < combos.size(); ++c)
        if (combos[c].l1 == l1 && combos[c].l2 == l2 && combos[c].m == mm && combos[c].part == part) return (int)c;
      combos.push_back(SCombo{l1, l2, mm, part});
      return (int)combos.size() - 1;
    };
    std::vector<std::vector<std::pair<int, double>>> terms(sug->nmult);
    for (int e = 0; !sugi_ep && e < sug->nmult; ++e) {
      const int l1 = sug->l1[e], l2 = sug->l2[e], L = sug->L[e], mmax = std::min(l1, l2);
      const double hN = wigner3j_host(l1, l2, L, 0, 0, 0) * (2 * l1 + 1) * (2 * l2 + 1) * (2 * L + 1);
      for (int mm = -mmax; mm <= mmax; ++mm) {
        const double w = hN * wigner3j_host(l1, l2, L, mm, -mm, 0) * (((l2 + mm) & 1) ? -1.0 : 1.0);
        const int am = std::abs(mm);
        for (int part = 0; part < 2; ++part) {
          if (am == 0 && part == ((l1 & 1) ? 0 : 1)) continue;   // the vanishing part at m = 0
          terms[e].push_back({combo_of(l1, l2, am, part), w});
        }
      }
    }
    if (!sugi_ep) {
      scoef.assign((size_t)sug->nmult * combos.size(), 0.0);
      for (int e = 0; e < sug->nmult; ++e)
        for (const auto& tw : terms[e]) scoef[(size_t)e * combos.size() + tw.first] += tw.second;
    }
    // rows b: A = the l1 part of bin b, B = G (pair (b, 0)); columns: the l2 parts of every bin
    std::vector<int> sp(nb);
    for (int b = 0; b < nb; ++b) sp[b] = b;
    t_spij = push_bytes(sp.data(), sizeof(int) * nb);
    t_srow = push_bytes(sp.data(), sizeof(int) * nb);
    t_scoef = push_bytes(scoef.data(), sizeof(double) * scoef.size());
    std::vector<double> sdesc((size_t)sug->nmult * SUGI_DESC, 0.0);
    for (int e = 0; e < sug->nmult; ++e) {
      const int l1 = sug->l1[e], l2 = sug->l2[e], L = sug->L[e];
      double* dd = sdesc.data() + (size_t)e * SUGI_DESC;
      dd[0] = l1;
      dd[1] = l2;
      dd[2] = L;
      dd[3] = wigner3j_host(l1, l2, L, 0, 0, 0) * (2 * l1 + 1) * (2 * l2 + 1) * (2 * L + 1);
      for (int n = -4; n <= 4; ++n) dd[4 + n + 4] = wigner3j_host(l1, l2, L, n, -n, 0);
    }
    t_sdesc = push_bytes(sdesc.data(), sizeof(double) * sdesc.size());
  }
  char* dtab;
  NPC_TRY(ws_table(ctx, need_nt ? "bis.tables.nt" : "bis.tables", tables, tables.data(), tables.size(),
                   (void**)&dtab));
  const ShellField* dfields = (const ShellField*)(dtab + t_fields);
  C *T1, *T2;
  T* R;
  NPC_TRY(ws_get(ctx, "bis.T1", sizeof(C) * std::max<int64_t>(o1, 1), (void**)&T1));
  NPC_TRY(ws_get(ctx, "bis.T2", sizeof(C) * std::max<int64_t>(o2, 1), (void**)&T2));
  // float fields chunk-interleaved (rf_index), float64 fields one row each
  const size_t rbytes = sizeof(T) * ncs * nfield;
  if (sizeof(T) == 4 && ncs % RCH != 0) return set_err(ctx, NPC_ERR_UNSUPPORTED, "shell grid of %lld cells", (long long)ncs);
  NPC_TRY(ws_get(ctx, "bis.R", rbytes, (void**)&R));
  const int16_t* tab_shell;
  NPC_TRY(get_bin_table(ctx, N, m.box, kb, &tab_shell, 2));
  unsigned* fmax_dev = nullptr;
  {
    ShellLaunch sl{};
    sl.X = X;
    sl.XN = fftshot ? (const void*)(X + xfs) : nullptr;
    sl.X2 = yam ? (const void*)(X + 2 * xfs) : nullptr;
    sl.X1 = (yamo && want1) ? (const void*)(X + 4 * xfs) : nullptr;
    sl.X3 = (yamo && want3) ? (const void*)(X + 5 * xfs) : nullptr;
    sl.XB = crq ? (const void*)(X + xfs) : nullptr;
    sl.XC = crq ? (const void*)(X + 2 * xfs) : nullptr;
    sl.XCOMP = sugi_ep ? (const void*)X : nullptr;
    sl.KZX = KZ;
    sl.nfine = N;
    sl.fields = dfields;
    sl.nfield = nfield;
    sl.Kmax = Kshell;
    sl.tab = tab_shell;
    sl.n2cap = n2cap;
    sl.frame = frame;
    sl.has_yw = sugi ? 1 : 0;
    sl.plane_f = (const int*)(dtab + t_pf);
    sl.plane_kz = (const int*)(dtab + t_pk);
    sl.nplanes = (int)plane_f.size();
    sl.za = (const int*)(dtab + t_za);
    sl.zb = (const int*)(dtab + t_zb);
    sl.oa = (const int*)(dtab + t_oa);
    sl.ob = (const int*)(dtab + t_ob);
    sl.nzp = nzp;
    sl.fmax = nullptr;
    if constexpr (sizeof(T) == 4) if (ctx->use_tcgen05 && !sugi) {
      NPC_TRY(ws_get(ctx, "bis.fmax", sizeof(unsigned) * nfield, (void**)&sl.fmax));
      NPC_CUDA(ctx, cudaMemsetAsync(sl.fmax, 0, sizeof(unsigned) * nfield, ctx->stream));
      fmax_dev = sl.fmax;
    }
    NPC_TRY(shell_dispatch<T>(ctx, NS, sl, T1, T2, R));
  }
  NPC_TRY(stage_mark(ctx, "shell_fields"));

  // 5. triple products
  if (nb > NB_MAX) return set_err(ctx, NPC_ERR_UNSUPPORTED, "at most %d bins", NB_MAX);
  int fam_of_l[4] = {0, -1, -1, -1};   // row family of B_l in the data launch
  auto setup = [&](TripleArgs& a, bool indicator) {
    a = TripleArgs{};
    a.npair = npair;
    a.ncell = (int64_t)ncs;
    a.nstage = 0;
    auto stage_of = [&](int field) {
      for (int q = 0; q < a.nstage; ++q)
        if (a.stage_field[q] == field) return q;
      a.stage_field[a.nstage] = field;
      return a.nstage++;
    };
    for (int q = 0; q < TRI_COLS; ++q) a.c_slot[q] = -1;
    a.nf_cols = nb;
    if (indicator) {
      for (int b = 0; b < nb; ++b) a.a_slot[0][b] = a.b_slot[0][b] = a.b_slot[1][b] = a.c_slot[b] = stage_of(iI + b);
      a.nrows = npair;
      a.ncol = nb;
    } else {
      for (int b = 0; b < nb; ++b) {
        a.a_slot[0][b] = stage_of(b);
        a.b_slot[0][b] = stage_of(iFB + b);
        a.c_slot[b] = stage_of(iFC + b);
      }
      // further row families: A = F_l (l = 2, 1, 3 as requested), B = F_0
      int nfam = 1;
      auto family_rows = [&](int first) {
        for (int b = 0; b < nb; ++b) {
          a.a_slot[nfam][b] = stage_of(first + b);
          a.b_slot[nfam][b] = stage_of(iFB + b);
        }
        return nfam++;
      };
      if (want2) fam_of_l[2] = family_rows(iF2);
      if (iFodd[1] >= 0) fam_of_l[1] = family_rows(iFodd[1]);
      if (iFodd[3] >= 0) fam_of_l[3] = family_rows(iFodd[3]);
      for (int l = 0; l < ng; ++l) a.c_slot[nb + l] = stage_of(iG + l);
      a.nrows = npair * nfam;
      a.ncol = nb + ng;
    }
  };
  TripleArgs ta, tn;
  setup(ta, false);
  setup(tn, true);
  // FFT-method shot noise products: rows (A_a, I_b) over pairs a <= b, columns over bins
  auto setup_shot = [&](TripleArgs& a, int fieldA0, int fieldA1, int fieldC) {
    a = TripleArgs{};
    a.npair = npair;
    a.ncell = (int64_t)ncs;
    a.nstage = 0;
    auto stage_of = [&](int field) {
      for (int q = 0; q < a.nstage; ++q)
        if (a.stage_field[q] == field) return q;
      a.stage_field[a.nstage] = field;
      return a.nstage++;
    };
    for (int q = 0; q < TRI_COLS; ++q) a.c_slot[q] = -1;
    for (int b = 0; b < nb; ++b) {
      a.a_slot[0][b] = stage_of(fieldA0 + b);
      a.b_slot[0][b] = a.b_slot[1][b] = stage_of(iI + b);
      a.c_slot[b] = stage_of(fieldC + b);
    }
    if (fieldA1 >= 0)
      for (int b = 0; b < nb; ++b) a.a_slot[1][b] = stage_of(fieldA1 + b);
    a.nf_cols = nb;
    a.nrows = npair * (fieldA1 >= 0 ? 2 : 1);
    a.ncol = nb;
  };
  TripleArgs ts1{}, ts2{}, tn2{}, ts3{};
  if (fftshot && !sugi) {
    setup_shot(ts1, iI, want2 ? iI2 : -1, iS0);   // sum I_a I_b S0_c and sum I2_a I_b S0_c
    if (ntl > 0) {
      // compressed estimator, same I_a I_b rows: columns nb + e: sum I_a I_b SF_l (Ta),
      // nb + ntl + e: sum I_a I_b LF_l (Td)
      auto stage_of = [&](int field) {
        for (int q = 0; q < ts1.nstage; ++q)
          if (ts1.stage_field[q] == field) return q;
        ts1.stage_field[ts1.nstage] = field;
        return ts1.nstage++;
      };
      for (int e = 0; e < ntl; ++e) {
        ts1.c_slot[nb + e] = stage_of(iSF + e);
        ts1.c_slot[nb + ntl + e] = stage_of(iLF + e);
      }
      ts1.ncol = nb + 2 * ntl;
      // rows (I_a, S0_b) and (S0_a, I_b), columns LF_l: Tb and Tc
      ts3 = TripleArgs{};
      ts3.npair = npair;
      ts3.ncell = (int64_t)ncs;
      auto stage3 = [&](int field) {
        for (int q = 0; q < ts3.nstage; ++q)
          if (ts3.stage_field[q] == field) return q;
        ts3.stage_field[ts3.nstage] = field;
        return ts3.nstage++;
      };
      for (int q = 0; q < TRI_COLS; ++q) ts3.c_slot[q] = -1;
      for (int b = 0; b < nb; ++b) {
        ts3.a_slot[0][b] = ts3.b_slot[1][b] = stage3(iI + b);
        ts3.b_slot[0][b] = ts3.a_slot[1][b] = stage3(iS0 + b);
      }
      for (int e = 0; e < ntl; ++e) ts3.c_slot[e] = stage3(iLF + e);
      ts3.nf_cols = 0;
      ts3.nrows = 2 * npair;
      ts3.ncol = ntl;
    }
    if (want2) setup_shot(ts2, iI, -1, iS2);      // sum I_a I_b S2_c
    if (want2) setup_shot(tn2, iI2, -1, iI);      // sum I2_a I_b I_c (cached)
  }
  // tensor-core (tcgen05) plans of the launches with more than 32 rows, one device table for all
  std::vector<std::pair<const TripleArgs*, TcPlanHost>> tc_plans;
  const char* tc_tab = nullptr;
  if constexpr (sizeof(T) == 4) {
    if (ctx->use_tcgen05 && fmax_dev) {
      int max_smem = 0;
      NPC_CUDA(ctx, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
      std::vector<char> tt;
      auto push16 = [&](const void* q, size_t nbytes) {
        const size_t o = tt.size();
        tt.resize(o + (nbytes + 15) / 16 * 16);
        if (nbytes) std::memcpy(tt.data() + o, q, nbytes);
        return o;
      };
      // the data and N_T launches are read only at the closed triangles (i <= j <= k: pair (i, j),
      // column k) and, for the data launch, at every pair's G columns: product rows that serve no
      // closed triangle are not formed
      std::vector<char> need_pk((size_t)npair * nb, 0);
      {
        std::vector<int> pidx((size_t)nb * nb, -1);
        for (int q = 0; q < npair; ++q) pidx[(size_t)(tr.pij[q] & 0xffff) * nb + (tr.pij[q] >> 16)] = q;
        for (size_t t = 0; t + 2 < tr.tri.size(); t += 3) {
          const int q = pidx[(size_t)tr.tri[t] * nb + tr.tri[t + 1]];
          if (q >= 0) need_pk[(size_t)q * nb + tr.tri[t + 2]] = 1;
        }
      }
      for (const TripleArgs* a : {&ta, &tn, &ts1, &ts2, &ts3, &tn2}) {
        TcPlanHost P;
        const std::vector<char>* need = (a == &ta || a == &tn) && a->nf_cols == nb ? &need_pk : nullptr;
        if (a->nrows <= 32 || a->ncol <= 0 || !plan_triple_tc(*a, tr.pij.data(), max_smem, P, need)) continue;
        P.o_rx = push16(P.rx.data(), sizeof(int16_t) * P.rx.size());
        P.o_ry = push16(P.ry.data(), sizeof(int16_t) * P.ry.size());
        P.o_cz = push16(P.cz.data(), sizeof(int16_t) * P.cz.size());
        P.o_sfield = push16(P.sfield.data(), sizeof(int) * P.sfield.size());
        P.o_runs = push16(P.runs.data(), sizeof(int) * P.runs.size());
        P.o_gidx = push16(P.gidx.data(), sizeof(int) * P.gidx.size());
        tc_plans.emplace_back(a, std::move(P));
      }
      if (!tc_plans.empty()) {
        void* d;
        NPC_TRY(ws_table(ctx, "bis.tcplan", tt, tt.data(), tt.size(), &d));
        tc_tab = (const char*)d;
      }
    }
  }
  auto tc_plan_of = [&](const TripleArgs& a) -> const TcPlanHost* {
    for (const auto& e : tc_plans)
      if (e.first == &a) return &e.second;
    return nullptr;
  };
  // one m tile per warp (3 CTAs per SM) while the staged fields leave room for three CTAs; the
  // tensor-core path: one CTA per SM and row group
  auto tri_mt = [&](const TripleArgs& a) { return a.nstage <= 47 ? 1 : 2; };
  auto grid_for = [&](const TripleArgs& a) {
    if (const TcPlanHost* P = tc_plan_of(a)) return std::max(1, ctx->num_sms / P->groups);
    const int mt = tri_mt(a), rows = TRI_WARPS * mt * 16;
    const int ng_ = (a.nrows + rows - 1) / rows;
    return sizeof(T) == 4 ? std::max(1, (mt == 1 ? 3 : 2) * ctx->num_sms / ng_) : ctx->num_sms * 4;
  };
  const int grid = grid_for(ta);
  double* part;
  NPC_TRY(ws_get(ctx, "bis.tripart", sizeof(double) * (size_t)grid * std::max(ta.nrows, tn.nrows) * TRI_COLS,
                 (void**)&part));
  auto launch_tab = [&](const TripleArgs& a0, int grid, double* part, size_t tp, size_t trp) -> npc_status {
    const TripleArgs& a = a0;
    TripleArgs ak = a0;   // the mma.sync path reads the float fields through rf_index
    ak.nfield_r = nfield;
    ctx->contraction_flops += 2.0 * a.nrows * a.ncol * (double)a.ncell;
    ctx->contraction_launches += 1;
    if constexpr (sizeof(T) == 4) {
      if (const TcPlanHost* P = tc_plan_of(a)) {
        // tensor-core (tcgen05) path, f16 hi + lo operands, orientation from the plan
        tc::Plan kp{};
        kp.nmrow = P->nmrow;
        kp.nmcol = P->nmcol;
        kp.n = P->n;
        kp.nsa = P->nsa;
        kp.nout = a.nrows * a.ncol;
        kp.nstage = a.nstage;
        kp.nrun = (int)P->runs.size() / 2;
        kp.nfield = nfield;
        kp.rx = (const int16_t*)(tc_tab + P->o_rx);
        kp.ry = (const int16_t*)(tc_tab + P->o_ry);
        kp.cz = (const int16_t*)(tc_tab + P->o_cz);
        kp.sfield = (const int*)(tc_tab + P->o_sfield);
        kp.runs = (const int*)(tc_tab + P->o_runs);
        kp.gidx = (const int*)(tc_tab + P->o_gidx);
        auto go = [&](auto kern) -> npc_status {
          NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->smem));
          kern<<<dim3(grid, P->groups), P->nt * 128 * tc::PPR + (tc::NBW + 2) * 32, P->smem, ctx->stream>>>(
              (const float*)R, a.ncell, kp, fmax_dev, part, ctx->dev_status, wait_cycles(ctx), P->nbuf);
          return NPC_OK;
        };
        NPC_TRY(P->nt == 1 ? go(k_triple_tc<1>) : P->nt == 2 ? go(k_triple_tc<2>) : go(k_triple_tc<3>));
        ctx->contraction_issued_flops += 2.0 * 2.0 * P->groups * P->nt * 128.0 * P->n * (double)a.ncell;
        ctx->bounded_waits = true;
        NPC_LAUNCH(ctx);
        return NPC_OK;
      }
      const int mt = tri_mt(a), rows = TRI_WARPS * mt * 16;
      const int groups = (a.nrows + rows - 1) / rows;
      auto run = [&](auto kern, int nt) -> npc_status {
        const size_t smem = sizeof(float) * (size_t)a.nstage * TRI_SPAD +
                            sizeof(double) * (size_t)TRI_WARPS * 32 * mt * nt * 4;
        NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<dim3(grid, groups), TRI_WARPS * 32, smem, ctx->stream>>>(
            (const float*)R, ak, (const int*)(dtab + tp), (const int*)(dtab + trp), part);
        return NPC_OK;
      };
      // issued: three tf32 products per useful one, on 16-row m tiles and 8-column n tiles
      ctx->contraction_issued_flops +=
          3.0 * 2.0 * (a.nrows <= 32 && a.ncol <= 24 ? 32 : groups * rows) * (a.ncol <= 24 ? 24 : 32) * (double)a.ncell;
      if (a.nrows <= 32 && a.ncol <= 24) {
        // few rows: all warps on the same two m tiles, each on its own cells
        const size_t smem = sizeof(float) * (size_t)a.nstage * TRI_SPAD + sizeof(double) * (size_t)TRI_WARPS * 32 * 2 * 3 * 4;
        auto kern = k_triple<3, 2, true>;
        NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<dim3(grid, 1), TRI_WARPS * 32, smem, ctx->stream>>>((const float*)R, ak, (const int*)(dtab + tp),
                                                                   (const int*)(dtab + trp), part);
      } else if (a.ncol <= 24) {
        NPC_TRY(mt == 1 ? run(k_triple<3, 1>, 3) : run(k_triple<3, 2>, 3));
      } else {
        NPC_TRY(mt == 1 ? run(k_triple<4, 1>, 4) : run(k_triple<4, 2>, 4));
      }
    } else {
      const int outs = a.nrows * a.ncol;
      ctx->contraction_issued_flops += 2.0 * outs * (double)a.ncell;
      k_triple_f64<<<dim3(grid, (outs + 255) / 256), 256, 0, ctx->stream>>>((const double*)R, a,
                                                                             (const int*)(dtab + tp), part);
      (void)trp;
    }
    NPC_LAUNCH(ctx);
    return NPC_OK;
  };
  auto launch = [&](const TripleArgs& a, int grid, double* part) { return launch_tab(a, grid, part, t_pij, t_rowp); };
  if (sugi) {
    // one product per combination: rows F_l1^m part (bin i) x G, columns F_l2^m part (bin j)
    // (FFT-method shot noise: the same products of the indicator parts against X N^*, rows ncombo..)
    const int ncombo = (int)combos.size();
    const int nprod = fftshot ? 2 * ncombo : ncombo;
    std::vector<TripleArgs> targs(nprod);
    for (int c = 0; c < nprod; ++c) {
      TripleArgs& a = targs[c];
      a = TripleArgs{};
      a.npair = nb;
      a.ncell = (int64_t)ncs;
      auto stage_of = [&](int field) {
        for (int q = 0; q < a.nstage; ++q)
          if (a.stage_field[q] == field) return q;
        a.stage_field[a.nstage] = field;
        return a.nstage++;
      };
      for (int q = 0; q < TRI_COLS; ++q) a.c_slot[q] = -1;
      const SCombo& cb = combos[c % ncombo];
      const bool ind = c >= ncombo;
      const int fa = ind ? ifield[cb.l1][cb.m][cb.part] : (cb.fa >= 0 ? cb.fa : sfield[cb.l1][cb.m][cb.part]);
      const int fc = ind ? ifield[cb.l2][cb.m][cb.part] : (cb.fc >= 0 ? cb.fc : sfield[cb.l2][cb.m][cb.part]);
      for (int b = 0; b < nb; ++b) a.a_slot[0][b] = stage_of(fa + b);
      a.b_slot[0][0] = stage_of(ind ? iXN : (cb.fg >= 0 ? cb.fg : iG));
      for (int b = 0; b < nb; ++b) a.c_slot[b] = stage_of(fc + b);
      a.nf_cols = nb;
      a.nrows = nb;
      a.ncol = nb;
    }
    // float: the split-over-cells product with two CTAs per SM (few rows); float64: as the others
    const int gsug = sizeof(T) == 4 ? 2 * ctx->num_sms : grid_for(targs[0]);
    const size_t per = (size_t)gsug * nb * nb;
    double *spart, *sred;
    NPC_TRY(ws_get(ctx, "bis.sugpart", sizeof(double) * per * nprod, (void**)&spart));
    NPC_TRY(ws_get(ctx, "bis.sugred", sizeof(double) * (size_t)nb * nb * nprod, (void**)&sred));
    for (int c = 0; c < nprod; ++c) NPC_TRY(launch_tab(targs[c], gsug, spart + c * per, t_spij, t_srow));
    NPC_TRY(stage_mark(ctx, "triple"));
    for (int c = 0; c < nprod; ++c) {
      k_part_reduce<<<(nb * nb + 31) / 32, 32 * PR_SLICES, 0, ctx->stream>>>(spart + c * per, gsug, (int64_t)nb * nb,
                                                                            sred + (size_t)c * nb * nb);
      NPC_LAUNCH(ctx);
    }
    double* sbins = nullptr;
    if (fftshot) {
      // per-bin lattice sums A_l^m and C_l^m of the pair terms with a free third leg
      const int nrows = (K + 1) * (2 * K + 1);
      const int g = std::min(nrows, ctx->num_sms * 2);
      const size_t np = (size_t)g * (BT / 32);
      double* bpart;
      NPC_TRY(ws_get(ctx, "bis.sbpart", sizeof(double) * np * NSB * nb, (void**)&bpart));
      NPC_CUDA(ctx, cudaMemsetAsync(bpart, 0, sizeof(double) * np * NSB * nb, ctx->stream));
      NPC_TRY(ws_get(ctx, "bis.sbins", sizeof(double) * NSB * nb, (void**)&sbins));
      k_sugi_binsums<T, N><<<g, BT, 0, ctx->stream>>>(X, X + xfs, K, frame, tab_m, nb, bpart);
      NPC_LAUNCH(ctx);
      k_cross_reduce<<<(nb * NSB + 3) / 4, 128, 0, ctx->stream>>>(bpart, (int)np, nb, NSB, sbins);
      NPC_LAUNCH(ctx);
    }
    // one 32-thread block (a warp) per output: the shot-noise sums are float64 work, spread over the SMs
    k_sugi_finalize<<<std::max(1, sug->nmult * nb * nb), 32, 0, ctx->stream>>>(
        sred, ncombo, (const double*)(dtab + t_scoef), (const double*)(dtab + t_sdesc), sug->nmult, nb, cross_m,
        cross_q, nq, nsum_c, shot, sbins, kb.dk, kb.kmin, sc, (double)ncs, dev_out);
    NPC_LAUNCH(ctx);
    NPC_TRY(stage_mark(ctx, "finalize"));
    (void)out_len;
    return NPC_OK;
  }
  if (need_nt) {
    NPC_TRY(launch(tn, grid, part));
    k_nt_reduce<<<(npair * nb + 127) / 128, 128, 0, ctx->stream>>>(part, grid, npair, nb, nb, (double)ncs, 1,
                                                                  nt_sums);
    NPC_LAUNCH(ctx);
    ctx->host_cache_keys[ntname] = ntkey;
  }
  if (need_nt2) {
    const int g2 = grid_for(tn2);
    double* p2;
    NPC_TRY(ws_get(ctx, "bis.nt2part", sizeof(double) * (size_t)g2 * tn2.nrows * nb, (void**)&p2));
    NPC_TRY(launch(tn2, g2, p2));
    k_nt_reduce<<<(npair * nb + 127) / 128, 128, 0, ctx->stream>>>(p2, g2, npair, nb, nb, (double)ncs, 0,
                                                                  nt2_sums);
    NPC_LAUNCH(ctx);
    ctx->host_cache_keys[nt2name] = nt2key;
  }
  NPC_TRY(launch(ta, grid, part));
  NPC_TRY(stage_mark(ctx, "triple"));
  double *part_s1 = nullptr, *part_s2 = nullptr, *part_s3 = nullptr;
  int gs1 = 0, gs2 = 0, gs3 = 0;
  if (fftshot) {
    gs1 = grid_for(ts1);
    NPC_TRY(ws_get(ctx, "bis.s1part", sizeof(double) * (size_t)gs1 * ts1.nrows * ts1.ncol, (void**)&part_s1));
    NPC_TRY(launch(ts1, gs1, part_s1));
    if (want2) {
      gs2 = grid_for(ts2);
      NPC_TRY(ws_get(ctx, "bis.s2part", sizeof(double) * (size_t)gs2 * ts2.nrows * nb, (void**)&part_s2));
      NPC_TRY(launch(ts2, gs2, part_s2));
    }
    if (ntl > 0) {
      gs3 = grid_for(ts3);
      NPC_TRY(ws_get(ctx, "bis.s3part", sizeof(double) * (size_t)gs3 * ts3.nrows * ts3.ncol, (void**)&part_s3));
      NPC_TRY(launch(ts3, gs3, part_s3));
    }
    NPC_TRY(stage_mark(ctx, "shot_triple"));
  }

  // 6. finalize: the per-CTA partials are summed first (one coalesced pass each), then combined
  auto reduce_parts = [&](const char* name, const double* p, int nparts, int64_t nent, double** out) -> npc_status {
    NPC_TRY(ws_get(ctx, name, sizeof(double) * std::max<int64_t>(nent, 1), (void**)out));
    const int64_t blocks = (nent + 31) / 32;
    if (blocks > INT32_MAX) return NPC_ERR_INVALID_ARG;
    k_part_reduce<<<(unsigned)std::max<int64_t>(1, blocks), 32 * PR_SLICES, 0, ctx->stream>>>(p, nparts, nent, *out);
    NPC_LAUNCH(ctx);
    return NPC_OK;
  };
  double *red_main = nullptr, *red_s1 = nullptr, *red_s2 = nullptr, *red_s3 = nullptr;
  NPC_TRY(reduce_parts("bis.red.main", part, grid, (int64_t)ta.nrows * ta.ncol, &red_main));
  if (fftshot) {
    NPC_TRY(reduce_parts("bis.red.s1", part_s1, gs1, (int64_t)ts1.nrows * ts1.ncol, &red_s1));
    if (want2) NPC_TRY(reduce_parts("bis.red.s2", part_s2, gs2, (int64_t)ts2.nrows * nb, &red_s2));
    if (ntl > 0) NPC_TRY(reduce_parts("bis.red.s3", part_s3, gs3, (int64_t)ts3.nrows * ts3.ncol, &red_s3));
  }
  FinalArgs fa{};
  fa.nb = nb;
  fa.ntri = ntri;
  fa.npair = npair;
  fa.nq = nq;
  fa.nscoc = 0;
  for (int l = 0; l <= 3; ++l)
    if (scoc_mask & (1 << l)) {
      fa.scoc_fam[fa.nscoc] = fam_of_l[l];
      fa.scoc_l[fa.nscoc++] = l;
    }
  fa.ntripo = 0;
  for (int l = 0; l <= 2; l += 2)
    if (tripo_mask & (1 << l)) fa.tripo_l[fa.ntripo++] = l;
  fa.shot = shot;
  fa.nparts = 1;   // partials already summed over the CTAs
  fa.nrows = ta.nrows;
  fa.ncol = ta.ncol;
  fa.ncell = (int64_t)ncs;
  fa.kmin = kb.kmin;
  fa.dk = kb.dk;
  fa.s1_nparts = gs1 > 0 ? 1 : 0;
  fa.s1_nrows = ts1.nrows;
  fa.s1_ncol = ts1.ncol;
  fa.s2_nparts = gs2 > 0 ? 1 : 0;
  fa.s2_nrows = ts2.nrows;
  fa.survey = yam ? 1 : 0;
  fa.ncs = nsum_c;
  fa.s3_nparts = gs3 > 0 ? 1 : 0;
  fa.s3_nrows = ts3.nrows;
  fa.s3_ncol = ts3.ncol;
  fa.ntri_blocks = (std::max(std::max(ntri, nb), 8) + 31) / 32;
  k_bispec_finalize<<<fa.ntri_blocks + npair, 32, 0, ctx->stream>>>(
      (const int*)(dtab + t_tri), (const int*)(dtab + t_pij), red_main, nt_sums, cross_m, cross_q, mom, red_s1, red_s2,
      red_s3, nt2_sums, fa, sc, dev_out);
  NPC_LAUNCH(ctx);
  NPC_TRY(stage_mark(ctx, "finalize"));
  (void)out_len;
  return NPC_OK;
}

template <typename T>
npc_status bispec_dispatch(npc_ctx* ctx, const npc_mesh_spec& m, const npc_kbins& kb, int sm, int tm, int shot,
                           const DevCatalog& d, const DevCatalog* r, double* sc, double* out, int64_t len,
                           const SugiReq* sug = nullptr, const CrossReq* crq = nullptr, double* sc_own = nullptr) {
  switch (m.n) {
    case 16: return bispec_impl<T, 16>(ctx, m, kb, sm, tm, shot, d, r, sc, out, len, sug, crq, sc_own);
    case 32: return bispec_impl<T, 32>(ctx, m, kb, sm, tm, shot, d, r, sc, out, len, sug, crq, sc_own);
    case 64: return bispec_impl<T, 64>(ctx, m, kb, sm, tm, shot, d, r, sc, out, len, sug, crq, sc_own);
    case 128: return bispec_impl<T, 128>(ctx, m, kb, sm, tm, shot, d, r, sc, out, len, sug, crq, sc_own);
    case 256: return bispec_impl<T, 256>(ctx, m, kb, sm, tm, shot, d, r, sc, out, len, sug, crq, sc_own);
    case 48: return bispec_impl<T, 48>(ctx, m, kb, sm, tm, shot, d, r, sc, out, len, sug, crq, sc_own);
    case 96: return bispec_impl<T, 96>(ctx, m, kb, sm, tm, shot, d, r, sc, out, len, sug, crq, sc_own);
    case 192: return bispec_impl<T, 192>(ctx, m, kb, sm, tm, shot, d, r, sc, out, len, sug, crq, sc_own);
  }
  if constexpr (sizeof(T) == 4) {
    if (m.n == 512) return bispec_impl<T, 512>(ctx, m, kb, sm, tm, shot, d, r, sc, out, len, sug, crq, sc_own);
  }
  return set_err(ctx, NPC_ERR_UNSUPPORTED, "bispectrum mesh size %d not supported at this precision", m.n);
}

}  // namespace

npc_status run_bispectrum(npc_ctx* ctx, const npc_mesh_spec& m, const npc_kbins& kb, int scoc_mask, int tripo_mask,
                          int shot, int prec, const DevCatalog& d, const DevCatalog* r, double* sc, double* out,
                          int64_t len) {
  if (prec == NPC_PREC_FP64)
    return bispec_dispatch<double>(ctx, m, kb, scoc_mask, tripo_mask, shot, d, r, sc, out, len);
  return bispec_dispatch<float>(ctx, m, kb, scoc_mask, tripo_mask, shot, d, r, sc, out, len);
}

npc_status run_bispectrum_cross(npc_ctx* ctx, const npc_mesh_spec& m, const npc_kbins& kb, int scoc_mask,
                                int tripo_mask, int prec, const DevCatalog& d, const DevCatalog* r, double* sc1,
                                double* scx, const CrossReq& req, double* out, int64_t len) {
  if (prec == NPC_PREC_FP64)
    return bispec_dispatch<double>(ctx, m, kb, scoc_mask, tripo_mask, 0, d, r, scx, out, len, nullptr, &req, sc1);
  return bispec_dispatch<float>(ctx, m, kb, scoc_mask, tripo_mask, 0, d, r, scx, out, len, nullptr, &req, sc1);
}

npc_status run_bispectrum_sugiyama(npc_ctx* ctx, const npc_mesh_spec& m, const npc_kbins& kb, const SugiReq& req,
                                   int shot, int prec, const DevCatalog& d, const DevCatalog* r, double* sc,
                                   double* out, int64_t len) {
  if (prec == NPC_PREC_FP64) return bispec_dispatch<double>(ctx, m, kb, 1, 0, shot, d, r, sc, out, len, &req);
  return bispec_dispatch<float>(ctx, m, kb, 1, 0, shot, d, r, sc, out, len, &req);
}

int64_t bispec_counts(const npc_kbins& kb, int64_t* ntri, int64_t* npair) {
  const Tri t = make_triangles(kb);
  *ntri = (int64_t)t.tri.size() / 3;
  *npair = (int64_t)t.pij.size();
  return 0;
}

npc_status bispec_triangles(const npc_kbins& kb, int32_t* tri, int64_t cap, int64_t* ntri) {
  const Tri t = make_triangles(kb);
  *ntri = (int64_t)t.tri.size() / 3;
  if (tri) {
    if (cap < *ntri) return NPC_ERR_INVALID_ARG;
    for (size_t i = 0; i < t.tri.size(); ++i) tri[i] = t.tri[i];
  }
  return NPC_OK;
}
