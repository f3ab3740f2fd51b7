// Mesh-level estimators and their adjoints: P_l(k) (global line of sight) and the equilateral
// Scoccimarro B_0(k, k, k) of a given periodic mesh delta(x), the vector-Jacobian products of both
// with respect to delta, and the adjoint of CIC/TSC mass assignment with respect to the particle
// positions and weights.
//
// With X(q) = sum_x delta(x) e^{-iq.x} / W(q) (Eq. compensation) and a global line of sight,
//   P_l(b)  = (2l+1)/(I22 N_b) sum_{q in b} L_l(qhat.los) |X(q)|^2 - delta_l0 N0     (Eq. pk_final)
//   B_0(b)  = sum_x F_b(x)^3 / (I33 sum_x I_b(x)^3),   F_b(x) = sum_{q in b} X(q) e^{iq.x},
//             I_b(x) = sum_{q in b} e^{iq.x}                                          (Eq. bi_sco)
// with I22, N0, I33 fixed by the catalogue.  P_l is bilinear in delta and B_0 trilinear, so for a
// loss L with cotangents g_lb = dL/dP_l(b) and h_b = dL/dB_0(b)
//   dL/ddelta(x) = sum_q [2 K(q) X(q) + sum_b c_b Phi_b(q) D_b(q)] / W(q) e^{iq.x},
//   K(q) = sum_{l,b} g_lb (2l+1) Phi_b(q) L_l(qhat.los) / (I22 N_b),
//   c_b  = 3 h_b / (I33 sum_x I_b^3),   D_b(q) = sum_x F_b(x)^2 e^{-iq.x}.
// (The paper does not differentiate its estimators; these are the exact derivatives of the
// expressions above.)
//
// Every spectrum lives in a compact k-space layout: rows (kz, ky) with 0 <= kz <= K and
// |ky| <= K, K the largest integer component any bin can reach, each row a full length-n line in
// kx.  Passes:
//   forward     z and y passes of power.cu on kz <= K, then k_adj_xfwd: x transform and 1/W per
//               compact row -> X (compact);
//   P_l         k_adj_pbins: per-bin sums of |X|^2 L_l(mu) (float64, warp partials in lane
//               order), k_adj_pfinal: normalisation and, for the adjoint, the K(q) coefficients;
//   shells      k_adj_rows_inv (masked rows, inverse x) -> k_adj_y_inv (inverse y, compact rows
//               in) -> k_adj_z (inverse z of two real fields per complex column).  The z pass
//               consumes each column in registers: it sums F^3 for B_0, or squares F and
//               transforms F^2 forward again for the adjoint, so no real field ever reaches HBM;
//   adjoint     k_adj_y_fwd (forward y, compact rows out) -> k_adj_rows_fwd_acc (forward x,
//               shell mask times c_b, fixed-order sum over bins) -> Y (compact);
//               k_adj_rows_inv on (Y + 2 K X)/W -> k_adj_y_inv -> k_adj_z writes dL/ddelta.
//   positions   k_paint_adjoint: per particle, the gradient mesh gathered at the 27 (TSC) or 8
//               (CIC) taps with the derivative of the assignment window.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "fft_core.cuh"

namespace {

constexpr int AT = 256;   // threads of the row kernels
constexpr int ANS = 5;    // sums per bin: modes, |k| (index units), |X|^2 L_0, L_2, L_4
constexpr int ADJ_MAX_FIELDS = 64;

enum : int8_t { SRC_BIN = 0, SRC_ONE = 1, SRC_GRAD = 2 };

struct AField {
  int8_t src;     // SRC_BIN: X on the modes of `bin`; SRC_ONE: 1 on them; SRC_GRAD: (Y + 2KX)/W
  int16_t bin;
  int K;          // rows kz <= K, |ky| <= K
  int64_t off1;   // compact-row buffer offset (complex elements): [kz][ky + K][x]
  int64_t off2;   // plane buffer offset (complex elements): [kz][y][x]
};

struct AFieldTable {
  int nf;
  AField f[ADJ_MAX_FIELDS];
};

template <typename T> __device__ __forceinline__ T wsinc(T a, int p) {
  const T s = a == T(0) ? T(1) : sin(a) / a;
  T r = s;
  for (int i = 1; i < p; ++i) r *= s;
  return r;
}

// Segmented sums over runs of equal `bin` in a warp; each run's tail lane adds its sums into the
// warp's own float64 partial, tails taken in lane order (no atomics: reproducible bit for bit).
template <typename T, int NS>
__device__ __forceinline__ void seg_add_ordered(int lane, int bin, const T (&vals)[NS], double* mypart) {
  const unsigned full = 0xffffffffu;
  const int pb = __shfl_up_sync(full, bin, 1);
  const bool head = (lane == 0) || (pb != bin);
  const unsigned heads = __ballot_sync(full, head);
  const int seg = __popc(heads & (full >> (31 - lane)));
  unsigned addm = 0;
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int off = 1 << st;
    const int os = __shfl_up_sync(full, seg, off);
    if (lane >= off && os == seg) addm |= 1u << st;
  }
  const bool last = (lane == 31) || ((heads >> (lane + 1)) & 1u);
  T x[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    x[s] = vals[s];
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const T y = __shfl_up_sync(full, x[s], 1 << st);
      if (addm & (1u << st)) x[s] += y;
    }
  }
  unsigned tails = __ballot_sync(full, last && bin >= 0);
  while (tails) {
    const int L = __ffs(tails) - 1;
    tails &= tails - 1;
    if (lane == L) {
#pragma unroll
      for (int s = 0; s < NS; ++s) mypart[(size_t)bin * NS + s] += (double)x[s];
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------------
// forward x pass: H[kz][ky][x] (kz <= K planes) -> X[r][kx] = FFT_x / W for compact rows r
// ------------------------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(AT)
k_adj_xfwd(const cplx<T>* __restrict__ H, int K, int assign, const cplx<T>* __restrict__ tw_g,
           cplx<T>* __restrict__ X) {
  using C = cplx<T>;
  constexpr int TPF = N / 8;
  constexpr int G = AT / TPF;
  constexpr int NP = row_pad_len<N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* bufs = tw + N;
  T* winv = reinterpret_cast<T*>(bufs + (size_t)G * NP);
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = tw_g[i];
  for (int i = tid; i <= N / 2; i += blockDim.x) winv[i] = T(1) / wsinc<T>(T(M_PI) * T(i) / T(N), assign);
  __syncthreads();
  const int g = tid / TPF, t = tid % TPF;
  const int nyr = 2 * K + 1;
  const int nrows = (K + 1) * nyr;
  for (int r0 = blockIdx.x * G; r0 < nrows; r0 += gridDim.x * G) {
    const int r = r0 + g;
    const bool live = r < nrows;
    const int kz = live ? r / nyr : 0;
    const int jy = live ? r % nyr - K : 0;
    const int ky = jy < 0 ? jy + N : jy;
    C v[8];
    const C* src = H + ((size_t)kz * N + ky) * N;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = live ? src[t + q * TPF] : cmk(T(0), T(0));
    fft_block<N, -1>(v, t, tw, RowView<C>{bufs + (size_t)g * NP}, RowSync<N, AT>::make(g));
    if (live) {
      const int aj = jy < 0 ? -jy : jy;
      const T wyz = winv[aj] * winv[kz];
      C* dst = X + (size_t)r * N;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int kx = t + q * TPF;
        const int i = kx < N / 2 ? kx : kx - N;
        const T w = i == -N / 2 ? T(0) : wyz * winv[i < 0 ? -i : i];
        dst[kx] = cscale(v[q], w);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// P_l bin sums over the compact spectrum (half spectrum: weight 2 for kz > 0)
// ------------------------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(AT)
k_adj_pbins(const cplx<T>* __restrict__ X, int K, const int16_t* __restrict__ bintab, int nb, double lx_d,
            double ly_d, double lz_d, double* __restrict__ part) {
  constexpr int NW = AT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* mypart = part + ((size_t)blockIdx.x * NW + warp) * nb * ANS;
  const T lx = (T)lx_d, ly = (T)ly_d, lz = (T)lz_d;
  const int nyr = 2 * K + 1;
  const int nrows = (K + 1) * nyr;
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int kz = r / nyr, jy = r % nyr - K;
    for (int jb = warp * 32; jb < N; jb += AT) {
      const int j = jb + lane;
      const int i = j < N / 2 ? j : j - N;
      const int n2 = i * i + jy * jy + kz * kz;
      int bin = -1;
      T vals[ANS];
#pragma unroll
      for (int s = 0; s < ANS; ++s) vals[s] = T(0);
      if (j < N && i != -N / 2 && n2 > 0) bin = bintab[n2];
      if (bin >= 0) {
        const cplx<T> x = X[(size_t)r * N + j];
        const T p2 = x.x * x.x + x.y * x.y;
        const T kk = sqrt(T(n2));
        const T mu = (T(i) * lx + T(jy) * ly + T(kz) * lz) / kk;
        const T m2 = mu * mu;
        const T w = kz > 0 ? T(2) : T(1);
        vals[0] = w;
        vals[1] = w * kk;
        vals[2] = w * p2;
        vals[3] = w * p2 * (T(1.5) * m2 - T(0.5));
        vals[4] = w * p2 * ((T(35) * m2 - T(30)) * m2 + T(3)) * T(0.125);
      }
      seg_add_ordered<T, ANS>(lane, bin, vals, mypart);
    }
  }
}

struct PFinal {
  int nb, nparts, nell;
  int ell[3];
  double i22, n0, kf;
  int want_out;
};

// Per bin: fixed-order sum of the warp partials; outputs k_eff, N_modes, P_l; for the adjoint the
// coefficients coef[e][b] = g_eb (2l+1)/(I22 N_b).
// One CTA per bin: thread t sums partials t, t + 256, ... in order, then a fixed tree.
__global__ void __launch_bounds__(256)
k_adj_pfinal(const double* __restrict__ part, PFinal F, const double* __restrict__ dldp,
             double* __restrict__ out, double* __restrict__ coef) {
  const int b = blockIdx.x;
  __shared__ double sh[ANS][256];
  double a[ANS] = {0, 0, 0, 0, 0};
  for (int p = threadIdx.x; p < F.nparts; p += blockDim.x)
    for (int k = 0; k < ANS; ++k) a[k] += part[((size_t)p * F.nb + b) * ANS + k];
  for (int k = 0; k < ANS; ++k) sh[k][threadIdx.x] = a[k];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int k = 0; k < ANS; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double s[ANS];
  for (int k = 0; k < ANS; ++k) s[k] = sh[k][0];
  const bool has = s[0] > 0;
  if (F.want_out) {
    out[b] = has ? F.kf * s[1] / s[0] : 0.0;
    out[F.nb + b] = s[0];
    for (int e = 0; e < F.nell; ++e) {
      const int l = F.ell[e];
      double v = 0;
      if (has) v = (2 * l + 1) / F.i22 * s[2 + l / 2] / s[0] - (l == 0 ? F.n0 : 0.0);
      out[(size_t)(2 + e) * F.nb + b] = v;
    }
  }
  if (coef)
    for (int e = 0; e < F.nell; ++e)
      coef[(size_t)e * F.nb + b] = has ? dldp[(size_t)e * F.nb + b] * (2 * F.ell[e] + 1) / (F.i22 * s[0]) : 0.0;
}

// ------------------------------------------------------------------------------------------
// Row pass, inverse x: for every compact row (kz, ky) of the outer radius KM and every field that
// reaches it, the masked (or gradient) row transformed back along x.
// ------------------------------------------------------------------------------------------
struct GradArgs {
  const void* Y;      // compact accumulated B_0 term or nullptr
  const double* coef; // [nell][nb] or nullptr
  int nell;
  int ell[3];
  int nb;
  double los[3];
};

// The shell fields are band-limited (|q_i| <= K per component), so their products F^2, F^3 are
// too (2K, 3K): sums over cells and the transforms of F^2 restricted to |q| <= K are exact on any
// grid of NS >= 3K + 1 points per axis, up to the factor (n/NS)^3.  The shell passes therefore run
// on the smallest supported NS (n itself for the final gradient), reading and writing the
// compact rows of the n grid.  Row kx' of the NS grid holds the integer frequency
// i = kx' (kx' < NS/2) or kx' - NS.
template <typename T, int NS>
__global__ void __launch_bounds__(AT)
k_adj_rows_inv(const cplx<T>* __restrict__ X, int KM, int nfine, const AFieldTable ft,
               const int16_t* __restrict__ bintab, const GradArgs ga, int assign, const cplx<T>* __restrict__ tw_g,
               cplx<T>* __restrict__ T1) {
  using C = cplx<T>;
  constexpr int TPF = NS / 8;
  constexpr int G = RowGroups<NS, AT>::G;
  constexpr int NP = row_pad_len<NS>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* xrow = tw + NS;
  C* grow = xrow + NS;
  C* bufs = grow + NS;
  int* binrow = reinterpret_cast<int*>(bufs + (size_t)RowGroups<NS, AT>::NBUF * NP);
  T* winv = reinterpret_cast<T*>(binrow + NS);       // 1/W per |i| of the n grid, |i| <= nfine/2
  const int tid = threadIdx.x;
  for (int i = tid; i < NS; i += blockDim.x) tw[i] = tw_g[i];
  for (int i = tid; i <= nfine / 2; i += blockDim.x) winv[i] = T(1) / wsinc<T>(T(M_PI) * T(i) / T(nfine), assign);
  const int g = tid / TPF, t = tid % TPF;
  const int nyr = 2 * KM + 1;
  const int nrows = (KM + 1) * nyr;
  const C* Y = reinterpret_cast<const C*>(ga.Y);
  bool any_grad = false;
  for (int f = 0; f < ft.nf; ++f) any_grad |= ft.f[f].src == SRC_GRAD;
  __syncthreads();
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int kz = r / nyr, jy = r % nyr - KM;
    const int ay = jy < 0 ? -jy : jy;
    for (int kx = tid; kx < NS; kx += blockDim.x) {
      const int i = kx < NS / 2 ? kx : kx - NS;
      const bool ok = i != -NS / 2 && i != -nfine / 2;
      const int fx = i < 0 ? i + nfine : i;       // position in the n-grid row
      const int n2 = i * i + jy * jy + kz * kz;
      const int bin = (ok && n2 > 0) ? bintab[n2] : -1;
      binrow[kx] = bin;
      const C x = (X && ok) ? X[(size_t)r * nfine + fx] : cmk(T(0), T(0));
      xrow[kx] = x;
      if (any_grad) {
        C gv = (Y && ok) ? Y[(size_t)r * nfine + fx] : cmk(T(0), T(0));
        if (ga.coef && bin >= 0) {
          const T kk = sqrt(T(n2));
          const T mu = (T(i) * T(ga.los[0]) + T(jy) * T(ga.los[1]) + T(kz) * T(ga.los[2])) / kk;
          const T m2 = mu * mu;
          T kq = T(0);
          for (int e = 0; e < ga.nell; ++e) {
            const int l = ga.ell[e];
            const T L = l == 0 ? T(1) : (l == 2 ? T(1.5) * m2 - T(0.5) : ((T(35) * m2 - T(30)) * m2 + T(3)) * T(0.125));
            kq += T(ga.coef[(size_t)e * ga.nb + bin]) * L;
          }
          gv = cadd(gv, cscale(x, T(2) * kq));
        }
        const T w = ok ? winv[i < 0 ? -i : i] * winv[ay] * winv[kz] : T(0);
        grow[kx] = cscale(gv, w);
      }
    }
    __syncthreads();
    for (int f0 = 0; f0 < ft.nf; f0 += G) {
      const int f = f0 + g;
      bool live = g < G && f < ft.nf;
      AField sf{};
      if (live) {
        sf = ft.f[f];
        live = kz <= sf.K && ay <= sf.K;
      }
      C v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int kx = t + q * TPF;
        C a = cmk(T(0), T(0));
        if (live) {
          if (sf.src == SRC_GRAD) a = grow[kx];
          else if (binrow[kx] == sf.bin) a = sf.src == SRC_BIN ? xrow[kx] : cmk(T(1), T(0));
        }
        v[q] = a;
      }
      fft_block<NS, +1>(v, t, tw, RowView<C>{bufs + (size_t)g * NP}, RowSync<NS, AT>::make(g));
      if (live) {
        C* dst = T1 + sf.off1 + ((size_t)kz * (2 * sf.K + 1) + (jy + sf.K)) * NS;
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[t + q * TPF] = v[q];
      }
    }
    __syncthreads();
  }
}

template <int N> struct ACol {
  static constexpr int TX = N >= 512 ? 8 : 16;
  static constexpr int THREADS = TX * N / 8;
};

// inverse y: plane p = (field, kz); compact rows |ky| <= K in, full y out ([kz][y][x])
template <typename T, int N>
__global__ void __launch_bounds__(ACol<N>::THREADS)
k_adj_y_inv(const cplx<T>* __restrict__ T1, const AFieldTable* __restrict__ ftp, const int2* __restrict__ planes,
            const cplx<T>* __restrict__ tw_g, cplx<T>* __restrict__ T2) {
  using C = cplx<T>;
  constexpr int TX = ACol<N>::TX;
  constexpr int TPF = N / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* work = tw + N;
  const int tid = threadIdx.x;
  const int c = tid % TX, t = tid / TX;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = tw_g[i];
  const int2 pl = planes[blockIdx.y];
  const AField sf = ftp->f[pl.x];
  const int kz = pl.y;
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

// forward y: full y in, compact rows |ky| <= K out
template <typename T, int N>
__global__ void __launch_bounds__(ACol<N>::THREADS)
k_adj_y_fwd(const cplx<T>* __restrict__ T2, const AFieldTable* __restrict__ ftp, const int2* __restrict__ planes,
            const cplx<T>* __restrict__ tw_g, cplx<T>* __restrict__ T1) {
  using C = cplx<T>;
  constexpr int TX = ACol<N>::TX;
  constexpr int TPF = N / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* work = tw + N;
  const int tid = threadIdx.x;
  const int c = tid % TX, t = tid / TX;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = tw_g[i];
  const int2 pl = planes[blockIdx.y];
  const AField sf = ftp->f[pl.x];
  const int kz = pl.y;
  const int x = blockIdx.x * TX + c;
  const C* src = T2 + sf.off2 + (size_t)kz * N * N + x;
  C v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = src[(size_t)(t + q * TPF) * N];
  __syncthreads();
  fft_block<N, -1>(v, t, tw, ColView<C>{work + c, TX});
  C* dst = T1 + sf.off1 + (size_t)kz * (2 * sf.K + 1) * N + x;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int yi = t + q * TPF;
    const int ky = yi < N / 2 ? yi : yi - N;
    if (ky >= -sf.K && ky <= sf.K) dst[(size_t)(ky + sf.K) * N] = v[q];
  }
}

enum { ZMODE_CUBE = 0, ZMODE_SQUARE_FWD = 1, ZMODE_WRITE = 2 };

// z columns of two real fields a, b (b may be absent): inverse transform of
//   c(kz) = A(kz) + i B(kz),  c(n - kz) = conj A(kz) + i conj B(kz)  (kz <= K_a resp. K_b)
// gives F_a = Re c(z), F_b = Im c(z).  Then, per mode:
//   CUBE        per-block float64 sums of F_a^3 and F_b^3 -> cube[field][block];
//   SQUARE_FWD  forward transform of F_a^2 + i F_b^2, split into the two half spectra and written
//               back in place for kz <= K_a, K_b;
//   WRITE       F_a written to the real mesh out[z][y][x].
template <typename T, int N>
__global__ void __launch_bounds__(ACol<N>::THREADS)
k_adj_z(cplx<T>* __restrict__ T2, const AFieldTable* __restrict__ ftp, const int2* __restrict__ pairs, int mode,
        const cplx<T>* __restrict__ tw_g, double* __restrict__ cube, T* __restrict__ out) {
  using C = cplx<T>;
  constexpr int TX = ACol<N>::TX;
  constexpr int TPF = N / 8;
  constexpr int NT = ACol<N>::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* work = tw + N;
  double* red = reinterpret_cast<double*>(work + N * TX);  // [2][NT/32]
  const int tid = threadIdx.x;
  const int c = tid % TX, t = tid / TX;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = tw_g[i];
  const int2 pr = pairs[blockIdx.z];
  const AField fa = ftp->f[pr.x];
  const bool hasb = pr.y >= 0;
  AField fb{};
  if (hasb) fb = ftp->f[pr.y];
  const int Ka = fa.K, Kb = hasb ? fb.K : -1;
  const int y = blockIdx.y, x = blockIdx.x * TX + c;
  const size_t plane = (size_t)N * N;
  const size_t cell0 = (size_t)y * N + x;
  C* A = T2 + fa.off2 + cell0;
  C* B = hasb ? T2 + fb.off2 + cell0 : nullptr;
  C v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int zi = t + q * TPF;
    C a = cmk(T(0), T(0)), b = cmk(T(0), T(0));
    if (zi <= Ka) a = A[(size_t)zi * plane];
    else if (N - zi <= Ka) a = cconj(A[(size_t)(N - zi) * plane]);
    if (zi <= Kb) b = B[(size_t)zi * plane];
    else if (N - zi <= Kb) b = cconj(B[(size_t)(N - zi) * plane]);
    v[q] = cmk(a.x - b.y, a.y + b.x);
  }
  __syncthreads();
  fft_block<N, +1>(v, t, tw, ColView<C>{work + c, TX});
  if (mode == ZMODE_WRITE) {
    T* o = out + cell0;
#pragma unroll
    for (int q = 0; q < 8; ++q) o[(size_t)(t + q * TPF) * plane] = v[q].x;
    return;
  }
  if (mode == ZMODE_CUBE) {
    T sa = T(0), sb = T(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      sa += v[q].x * v[q].x * v[q].x;
      sb += v[q].y * v[q].y * v[q].y;
    }
    double da = (double)sa, db = (double)sb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      da += __shfl_down_sync(0xffffffffu, da, o);
      db += __shfl_down_sync(0xffffffffu, db, o);
    }
    const int lane = tid & 31, w = tid >> 5;
    if (lane == 0) {
      red[w] = da;
      red[NT / 32 + w] = db;
    }
    __syncthreads();
    if (tid == 0) {
      double ra = 0, rb = 0;
      for (int k = 0; k < NT / 32; ++k) {
        ra += red[k];
        rb += red[NT / 32 + k];
      }
      const size_t nblk = (size_t)gridDim.x * gridDim.y;
      const size_t blk = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
      cube[(size_t)pr.x * nblk + blk] = ra;
      if (hasb) cube[(size_t)pr.y * nblk + blk] = rb;
    }
    return;
  }
  // SQUARE_FWD
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = cmk(v[q].x * v[q].x, v[q].y * v[q].y);
  fft_block<N, -1>(v, t, tw, ColView<C>{work + c, TX});
#pragma unroll
  for (int q = 0; q < 8; ++q) work[(t + q * TPF) * TX + c] = v[q];
  __syncthreads();
  const int Kmx = Ka > Kb ? Ka : Kb;
  for (int kz = t; kz <= Kmx; kz += TPF) {
    const C z1 = work[kz * TX + c];
    const C z2 = cconj(work[((N - kz) % N) * TX + c]);
    if (kz <= Ka) A[(size_t)kz * plane] = cscale(cadd(z1, z2), T(0.5));
    if (kz <= Kb) {
      const C d = csub(z1, z2);
      B[(size_t)kz * plane] = cmk(T(0.5) * d.y, T(-0.5) * d.x);
    }
  }
}

// fixed-order float64 sum of the per-block cube partials of each field
__global__ void k_adj_cube_reduce(const double* __restrict__ cube, size_t nblk, double* __restrict__ sums) {
  const int f = blockIdx.x;
  __shared__ double sh[256];
  double s = 0;
  for (size_t i = threadIdx.x; i < nblk; i += blockDim.x) s += cube[(size_t)f * nblk + i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[f] = sh[0];
}

// Triangle counts: on the NS grid sum_x I_b^3 = NS^3 * (number of closed (q1, q2, q3) in bin b), an
// exact integer when no triple aliases (3 K < NS); rounded to it and stored as the n-grid sum
// n^3 * count.
__global__ void k_adj_nt_store(const double* __restrict__ sums, int first, int nb, double ncell_s, double ncell,
                               double* __restrict__ nt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) nt[b] = rint(sums[first + b] / ncell_s) * ncell;
}

// B_0 = (n/NS)^3 sum_NS F^3 / (I33 sum_n I^3); N_T = sum_n I^3 / n^3
__global__ void k_adj_b0_final(const double* __restrict__ sums, const double* __restrict__ nt, int nb, double i33,
                               double scale, double ncell, double* __restrict__ out_b0, double* __restrict__ out_nt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  out_b0[b] = nt[b] > 0 ? scale * sums[b] / (i33 * nt[b]) : 0.0;
  out_nt[b] = nt[b] / ncell;
}

// c_b = 3 h_b / (I33 sum_n I^3), times (n/NS)^3 for transforms of F^2 taken on the NS grid
__global__ void k_adj_bcoef(const double* __restrict__ nt, const double* __restrict__ h, int nb, double i33,
                            double scale, double* __restrict__ cb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) cb[b] = nt[b] > 0 ? 3.0 * scale * h[b] / (i33 * nt[b]) : 0.0;
}

// Row pass, forward x with accumulation: Y[r][kx] (+)= sum_f c_f Phi_f(q) FFT_x(T1_f row), fields
// summed per group then over groups in a fixed order; rows of the NS grid are mapped back onto the
// n-grid rows of Y.
template <typename T, int NS>
__global__ void __launch_bounds__(AT)
k_adj_rows_fwd_acc(const cplx<T>* __restrict__ T1, int KM, int nfine, const AFieldTable ft,
                   const int16_t* __restrict__ bintab, const double* __restrict__ cb, const cplx<T>* __restrict__ tw_g,
                   cplx<T>* __restrict__ Y) {
  using C = cplx<T>;
  constexpr int TPF = NS / 8;
  constexpr int G = RowGroups<NS, AT>::G;
  constexpr int NP = row_pad_len<NS>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* acc = tw + NS;                     // [G][NS]
  C* bufs = acc + (size_t)G * NS;       // [NBUF][NP]
  int* binrow = reinterpret_cast<int*>(bufs + (size_t)RowGroups<NS, AT>::NBUF * NP);
  const int tid = threadIdx.x;
  for (int i = tid; i < NS; i += blockDim.x) tw[i] = tw_g[i];
  const int g = tid / TPF, t = tid % TPF;
  const int nyr = 2 * KM + 1;
  const int nrows = (KM + 1) * nyr;
  __syncthreads();
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int kz = r / nyr, jy = r % nyr - KM;
    const int ay = jy < 0 ? -jy : jy;
    for (int kx = tid; kx < NS; kx += blockDim.x) {
      const int i = kx < NS / 2 ? kx : kx - NS;
      const int n2 = i * i + jy * jy + kz * kz;
      binrow[kx] = (i != -NS / 2 && i != -nfine / 2 && n2 > 0) ? bintab[n2] : -1;
    }
    for (int i = tid; i < G * NS; i += blockDim.x) acc[i] = cmk(T(0), T(0));
    __syncthreads();
    for (int f0 = 0; f0 < ft.nf; f0 += G) {
      const int f = f0 + g;
      bool live = g < G && f < ft.nf;
      AField sf{};
      if (live) {
        sf = ft.f[f];
        live = kz <= sf.K && ay <= sf.K;
      }
      C v[8];
      const C* src = T1 + (live ? sf.off1 + ((size_t)kz * (2 * sf.K + 1) + (jy + sf.K)) * NS : 0);
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = live ? src[t + q * TPF] : cmk(T(0), T(0));
      fft_block<NS, -1>(v, t, tw, RowView<C>{bufs + (size_t)g * NP}, RowSync<NS, AT>::make(g));
      if (live) {
        const T c = (T)cb[sf.bin];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int kx = t + q * TPF;
          if (binrow[kx] == sf.bin) acc[(size_t)g * NS + kx] = cadd(acc[(size_t)g * NS + kx], cscale(v[q], c));
        }
      }
    }
    __syncthreads();
    for (int kx = tid; kx < nfine; kx += blockDim.x) {
      const int i = kx < nfine / 2 ? kx : kx - nfine;
      C s = cmk(T(0), T(0));
      if (i > -NS / 2 && i < NS / 2) {
        const int cx = i < 0 ? i + NS : i;
        s = acc[cx];
        for (int q = 1; q < G; ++q) s = cadd(s, acc[(size_t)q * NS + cx]);
      }
      Y[(size_t)r * nfine + kx] = s;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// Adjoint of mass assignment: per particle p with grid coordinate s_p = (x_p - origin) n/box,
//   dL/dx_p,a = w_p (n/box) sum_taps G(c) dW/ds_a,   dL/dw_p = sum_taps G(c) W(c - s_p).
// Tap decisions (floor) are taken in float64 exactly as in the forward assignment.
// ------------------------------------------------------------------------------------------
template <int ASSIGN, typename TP, typename TG>
__global__ void __launch_bounds__(256)
k_paint_adjoint(const TP* __restrict__ pos, const TP* __restrict__ w, int64_t np, int N, double o0, double o1,
                double o2, double inv_h, const TG* __restrict__ grad, TP* __restrict__ gpos, TP* __restrict__ gw) {
  constexpr int NTAP = ASSIGN == 3 ? 3 : 2;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    const double o[3] = {o0, o1, o2};
    int idx[3][NTAP];
    TG W[3][NTAP], dW[3][NTAP];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double s = ((double)pos[3 * p + a] - o[a]) * inv_h;
      const double i0 = ASSIGN == 3 ? floor(s + 0.5) : floor(s);
      const TG d = (TG)(s - i0);
      const long long base = (long long)i0 - (ASSIGN == 3 ? 1 : 0);
#pragma unroll
      for (int k = 0; k < NTAP; ++k) {
        long long c = (base + k) % N;
        if (c < 0) c += N;
        idx[a][k] = (int)c;
      }
      if (ASSIGN == 3) {
        const TG u = TG(0.5) - d, v = TG(0.5) + d;
        W[a][0] = TG(0.5) * u * u;
        W[a][1] = TG(0.75) - d * d;
        W[a][2] = TG(0.5) * v * v;
        dW[a][0] = -u;
        dW[a][1] = TG(-2) * d;
        dW[a][2] = v;
      } else {
        W[a][0] = TG(1) - d;
        W[a][1] = d;
        dW[a][0] = TG(-1);
        dW[a][1] = TG(1);
      }
    }
    TG gx = 0, gy = 0, gz = 0, gv = 0;
#pragma unroll
    for (int kz = 0; kz < NTAP; ++kz)
#pragma unroll
      for (int ky = 0; ky < NTAP; ++ky) {
        const TG* row = grad + ((size_t)idx[2][kz] * N + idx[1][ky]) * N;
        const TG wyz = W[1][ky] * W[2][kz];
        const TG dyz = dW[1][ky] * W[2][kz];
        const TG ydz = W[1][ky] * dW[2][kz];
#pragma unroll
        for (int kx = 0; kx < NTAP; ++kx) {
          const TG G = row[idx[0][kx]];
          gx += G * dW[0][kx] * wyz;
          gy += G * W[0][kx] * dyz;
          gz += G * W[0][kx] * ydz;
          gv += G * W[0][kx] * wyz;
        }
      }
    const double ww = w ? (double)w[p] : 1.0;
    gpos[3 * p + 0] = (TP)(ww * inv_h * (double)gx);
    gpos[3 * p + 1] = (TP)(ww * inv_h * (double)gy);
    gpos[3 * p + 2] = (TP)(ww * inv_h * (double)gz);
    if (gw) gw[p] = (TP)gv;
  }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
struct MeshJob {
  int n;
  int ell_mask;       // P_l requested (bits 0, 2, 4)
  int want_b0;
  int want_out;       // forward values
  double i22, n0, i33;
  const double* dldp; // device [nell][nb] or nullptr
  const double* dldb; // device [nb] or nullptr
  void* grad;         // device mesh or nullptr
  double* out;        // device output or nullptr
};

int outer_radius(int n, double box, const npc_kbins& kb) {
  const double kf = 2.0 * M_PI / box;
  const double kmax = kb.kmin + kb.nbins * kb.dk;
  const double r = std::floor(kmax / kf) + 1.0;
  return (int)std::max(1.0, std::min((double)(n / 2 - 1), r));
}

int bin_radius(double box, const npc_kbins& kb, int b, int KM) {
  const double kf = 2.0 * M_PI / box;
  const double edge = kb.kmin + (b + 1) * kb.dk;
  const double r = std::floor(edge / kf) + 1.0;
  return (int)std::max(1.0, std::min((double)KM, r));
}

template <typename T, int N>
npc_status row_grid(npc_ctx* ctx, const void* kern, size_t smem, int nrows, int rows_per_block, int* grid) {
  int per_sm = 0;
  NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  NPC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, AT, smem));
  if (per_sm < 1) return set_err(ctx, NPC_ERR_UNSUPPORTED, "row kernel does not fit on an SM (%zu B smem)", smem);
  const int need = (nrows + rows_per_block - 1) / rows_per_block;
  *grid = std::max(1, std::min(need, per_sm * ctx->num_sms));
  return NPC_OK;
}

// Shell pipeline for a field table on the NS grid: inverse x (rows of radius KM), inverse y, then
// the z pass in `mode`; for SQUARE_FWD also forward y and the accumulating forward x into Y.
template <typename T, int NS>
npc_status shell_pass(npc_ctx* ctx, const AFieldTable& ft, const std::string& tag, int KM, int nfine,
                      const cplx<T>* X, const int16_t* bintab, const GradArgs& ga, int assign, int mode,
                      double* cube_sums, const double* cb, cplx<T>* Yacc, T* out) {
  using C = cplx<T>;
  const void* twp;
  NPC_TRY(get_twiddles(ctx, NS, sizeof(T) == 8 ? NPC_PREC_FP64 : NPC_PREC_MIXED, &twp));
  const C* tw = (const C*)twp;
  // buffers and plane / pair tables
  int64_t n1 = 0, n2 = 0;
  AFieldTable t = ft;
  std::vector<int2> planes, pairs;
  for (int f = 0; f < t.nf; ++f) {
    const int K = t.f[f].K;
    t.f[f].off1 = n1;
    t.f[f].off2 = n2;
    n1 += (int64_t)(K + 1) * (2 * K + 1) * NS;
    n2 += (int64_t)(K + 1) * NS * NS;
    for (int kz = 0; kz <= K; ++kz) planes.push_back(make_int2(f, kz));
  }
  for (int f = 0; f < t.nf; f += 2) pairs.push_back(make_int2(f, f + 1 < t.nf ? f + 1 : -1));
  C *T1, *T2;
  NPC_TRY(ws_get(ctx, "adj.T1", sizeof(C) * n1, (void**)&T1));
  NPC_TRY(ws_get(ctx, "adj.T2", sizeof(C) * n2, (void**)&T2));
  std::vector<char> blob(sizeof(AFieldTable) + sizeof(int2) * (planes.size() + pairs.size()));
  std::memcpy(blob.data(), &t, sizeof(AFieldTable));
  std::memcpy(blob.data() + sizeof(AFieldTable), planes.data(), sizeof(int2) * planes.size());
  std::memcpy(blob.data() + sizeof(AFieldTable) + sizeof(int2) * planes.size(), pairs.data(),
              sizeof(int2) * pairs.size());
  void* dtab;
  NPC_TRY(ws_table(ctx, "adj.tab." + tag, blob, blob.data(), blob.size(), &dtab));
  const AFieldTable* dft = (const AFieldTable*)dtab;
  const int2* dplanes = (const int2*)((char*)dtab + sizeof(AFieldTable));
  const int2* dpairs = dplanes + planes.size();

  constexpr int G = RowGroups<NS, AT>::G;
  constexpr int NBUF = RowGroups<NS, AT>::NBUF;
  constexpr int NP = row_pad_len<NS>();
  const int nrows = (KM + 1) * (2 * KM + 1);
  {
    const size_t smem = sizeof(C) * (3 * NS + (size_t)NBUF * NP) + sizeof(int) * NS + sizeof(T) * (nfine / 2 + 2);
    auto kern = k_adj_rows_inv<T, NS>;
    int grid;
    NPC_TRY((row_grid<T, NS>(ctx, (const void*)kern, smem, nrows, 1, &grid)));
    kern<<<grid, AT, smem, ctx->stream>>>(X, KM, nfine, t, bintab, ga, assign, tw, T1);
    NPC_LAUNCH(ctx);
  }
  NPC_TRY(stage_mark(ctx, "shell_x_inv"));
  constexpr int TX = ACol<NS>::TX;
  const size_t csmem = sizeof(C) * (NS + (size_t)NS * TX);
  {
    auto kern = k_adj_y_inv<T, NS>;
    NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem));
    for (size_t p0 = 0; p0 < planes.size(); p0 += 65535) {
      const int np = (int)std::min<size_t>(65535, planes.size() - p0);
      kern<<<dim3(NS / TX, np), ACol<NS>::THREADS, csmem, ctx->stream>>>(T1, dft, dplanes + p0, tw, T2);
      NPC_LAUNCH(ctx);
    }
  }
  NPC_TRY(stage_mark(ctx, "shell_y_inv"));
  {
    const size_t zsmem = csmem + sizeof(double) * 2 * (ACol<NS>::THREADS / 32);
    auto kern = k_adj_z<T, NS>;
    NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsmem));
    double* cube = nullptr;
    const size_t nblk = (size_t)(NS / TX) * NS;
    if (mode == ZMODE_CUBE) NPC_TRY(ws_get(ctx, "adj.cube", sizeof(double) * nblk * t.nf, (void**)&cube));
    kern<<<dim3(NS / TX, NS, (unsigned)pairs.size()), ACol<NS>::THREADS, zsmem, ctx->stream>>>(T2, dft, dpairs, mode,
                                                                                             tw, cube, out);
    NPC_LAUNCH(ctx);
    if (mode == ZMODE_CUBE) {
      k_adj_cube_reduce<<<t.nf, 256, 0, ctx->stream>>>(cube, nblk, cube_sums);
      NPC_LAUNCH(ctx);
    }
  }
  NPC_TRY(stage_mark(ctx, mode == ZMODE_WRITE ? "grad_z_inv" : (mode == ZMODE_CUBE ? "shell_z_cube" : "shell_z_sq_fwd")));
  if (mode != ZMODE_SQUARE_FWD) return NPC_OK;
  {
    auto kern = k_adj_y_fwd<T, NS>;
    NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem));
    for (size_t p0 = 0; p0 < planes.size(); p0 += 65535) {
      const int np = (int)std::min<size_t>(65535, planes.size() - p0);
      kern<<<dim3(NS / TX, np), ACol<NS>::THREADS, csmem, ctx->stream>>>(T2, dft, dplanes + p0, tw, T1);
      NPC_LAUNCH(ctx);
    }
  }
  NPC_TRY(stage_mark(ctx, "shell_y_fwd"));
  {
    const size_t smem = sizeof(C) * (NS + (size_t)G * NS + (size_t)NBUF * NP) + sizeof(int) * NS;
    auto kern = k_adj_rows_fwd_acc<T, NS>;
    int grid;
    NPC_TRY((row_grid<T, NS>(ctx, (const void*)kern, smem, nrows, 1, &grid)));
    kern<<<grid, AT, smem, ctx->stream>>>(T1, KM, nfine, t, bintab, cb, tw, Yacc);
    NPC_LAUNCH(ctx);
  }
  NPC_TRY(stage_mark(ctx, "shell_x_fwd_acc"));
  return NPC_OK;
}

// the smallest compiled transform length >= need (and <= n; FP64 up to 256)
int shell_grid(int need, int n, bool fp64) {
  static const int sizes[] = {16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 1024};
  for (int s : sizes) {
    if (s > n || (fp64 && s > 256)) break;
    if (s >= need) return s;
  }
  return n;
}

template <typename T>
npc_status shell_dispatch(npc_ctx* ctx, int NS, const AFieldTable& ft, const std::string& tag, int KM, int nfine,
                          const cplx<T>* X, const int16_t* bintab, const GradArgs& ga, int assign, int mode,
                          double* cube_sums, const double* cb, cplx<T>* Yacc, T* out) {
#define NPC_SHELL(S) \
  case S: return shell_pass<T, S>(ctx, ft, tag, KM, nfine, X, bintab, ga, assign, mode, cube_sums, cb, Yacc, out);
  switch (NS) {
    NPC_SHELL(16) NPC_SHELL(32) NPC_SHELL(48) NPC_SHELL(64) NPC_SHELL(96) NPC_SHELL(128) NPC_SHELL(192) NPC_SHELL(256)
  }
  if constexpr (sizeof(T) == 4) {
    switch (NS) { NPC_SHELL(384) NPC_SHELL(512) NPC_SHELL(1024) }
  }
#undef NPC_SHELL
  return set_err(ctx, NPC_ERR_UNSUPPORTED, "shell grid %d not supported at this precision", NS);
}

template <typename T, int N>
npc_status mesh_impl(npc_ctx* ctx, const npc_mesh_spec& m, const npc_kbins& kb, int prec, const void* mesh,
                     const MeshJob& job) {
  using C = cplx<T>;
  const int nb = kb.nbins;
  const int KM = outer_radius(N, m.box, kb);
  const double ncell = (double)N * N * N;
  // grid of the B_0 shell passes: every shell lies inside |q_i| <= KB, products up to 3 KB
  int KB = 1;
  for (int b = 0; b < nb; ++b) KB = std::max(KB, bin_radius(m.box, kb, b, KM));
  const int NS = shell_grid(3 * KB + 1, N, sizeof(T) == 8);
  const double ncell_s = (double)NS * NS * NS;
  const void* twp;
  NPC_TRY(get_twiddles(ctx, N, prec, &twp));
  const C* tw = (const C*)twp;
  const int16_t* bintab;
  NPC_TRY(get_bin_table(ctx, N, m.box, kb, &bintab, 4));

  // 1. forward transform of the mesh on kz <= KM, compact rows, 1/W
  PowerPlan plan{};
  plan.n = N;
  plan.nphase = 1;
  plan.fl.nf = 1;
  plan.fl.f[0].phase = 0;
  plan.fl.f[0].ell = 0;
  plan.fl.f[0].m = 0;
  plan.fl.f[0].part = PART_ONE;
  plan.global_los = 1;
  plan.assign = m.assign;
  plan.kz_keep = KM + 1;
  const Geom g = make_geom(m);
  C *H, *X;
  const size_t nrows = (size_t)(KM + 1) * (2 * KM + 1);
  NPC_TRY(ws_get(ctx, "adj.H", sizeof(C) * (size_t)(KM + 1) * N * N, (void**)&H));
  NPC_TRY(ws_get(ctx, "adj.X", sizeof(C) * nrows * N, (void**)&X));
  NPC_TRY(run_forward_transforms(ctx, prec, plan, g, mesh, nullptr, H));
  constexpr int TPF = N / 8;
  constexpr int G = AT / TPF;
  constexpr int NP = row_pad_len<N>();
  {
    const size_t smem = sizeof(C) * (N + (size_t)G * NP) + sizeof(T) * (N / 2 + 2);
    auto kern = k_adj_xfwd<T, N>;
    int grid;
    NPC_TRY((row_grid<T, N>(ctx, (const void*)kern, smem, (int)nrows, G, &grid)));
    kern<<<grid, AT, smem, ctx->stream>>>(H, KM, m.assign, tw, X);
    NPC_LAUNCH(ctx);
  }
  NPC_TRY(stage_mark(ctx, "fft_x_fwd"));

  const Geom gl = g;
  int nell = 0, ells[3];
  for (int l = 0; l <= 4; l += 2)
    if (job.ell_mask & (1 << l)) ells[nell++] = l;

  // 2. P_l sums (forward values and/or the adjoint coefficients)
  double* coef = nullptr;
  const bool need_p = job.want_out || (nell > 0 && job.dldp);
  if (need_p) {
    const int grid = std::min<int>((int)nrows, 2 * ctx->num_sms);
    const size_t nparts = (size_t)grid * (AT / 32);
    double* part;
    NPC_TRY(ws_get(ctx, "adj.ppart", sizeof(double) * nparts * nb * ANS, (void**)&part));
    NPC_CUDA(ctx, cudaMemsetAsync(part, 0, sizeof(double) * nparts * nb * ANS, ctx->stream));
    k_adj_pbins<T, N><<<grid, AT, 0, ctx->stream>>>(X, KM, bintab, nb, gl.los[0], gl.los[1], gl.los[2], part);
    NPC_LAUNCH(ctx);
    PFinal F{};
    F.nb = nb;
    F.nparts = (int)nparts;
    F.nell = nell;
    for (int e = 0; e < nell; ++e) F.ell[e] = ells[e];
    F.i22 = job.i22;
    F.n0 = job.n0;
    F.kf = 2.0 * M_PI / m.box;
    F.want_out = job.want_out ? 1 : 0;
    if (job.dldp) NPC_TRY(ws_get(ctx, "adj.coef", sizeof(double) * nell * nb, (void**)&coef));
    k_adj_pfinal<<<nb, 256, 0, ctx->stream>>>(part, F, job.dldp, job.out, coef);
    NPC_LAUNCH(ctx);
    NPC_TRY(stage_mark(ctx, "power_bins"));
  }

  // 3. equilateral B_0: bin shells, triangle counts (cached per geometry)
  double* nt = nullptr;
  if (job.want_b0) {
    NPC_TRY(ws_get(ctx, slot_name(ctx, "adj.nt").c_str(), sizeof(double) * nb, (void**)&nt));
    std::vector<char> key;
    auto push = [&](const void* p, size_t s) { key.insert(key.end(), (const char*)p, (const char*)p + s); };
    const int nn = N;
    push(&nn, sizeof(nn));
    push(&m.box, sizeof(double));
    push(&kb, sizeof(kb));
    const int tsize = (int)sizeof(T);   // float and float64 shells round differently
    push(&tsize, sizeof(tsize));
    const std::string ntname = slot_name(ctx, "adj.nt");
    auto it = ctx->host_cache_keys.find(ntname);
    const bool nt_ok = it != ctx->host_cache_keys.end() && it->second == key;
    const bool fwd_b0 = job.want_out != 0;
    double* sums;
    NPC_TRY(ws_get(ctx, "adj.sums", sizeof(double) * 2 * nb, (void**)&sums));
    // forward values: F_b^3 sums (and the counts when not cached) in one shell pass
    if (fwd_b0 || !nt_ok) {
      AFieldTable ft{};
      ft.nf = 0;
      if (fwd_b0)
        for (int b = 0; b < nb; ++b) ft.f[ft.nf++] = AField{SRC_BIN, (int16_t)b, bin_radius(m.box, kb, b, KM), 0, 0};
      const int first_one = ft.nf;
      if (!nt_ok)
        for (int b = 0; b < nb; ++b) ft.f[ft.nf++] = AField{SRC_ONE, (int16_t)b, bin_radius(m.box, kb, b, KM), 0, 0};
      GradArgs ga{};
      NPC_TRY(shell_dispatch<T>(ctx, NS, ft, "cube", KM, N, X, bintab, ga, m.assign, ZMODE_CUBE, sums, nullptr,
                                nullptr, nullptr));
      if (!nt_ok) {
        k_adj_nt_store<<<(nb + 127) / 128, 128, 0, ctx->stream>>>(sums, first_one, nb, ncell_s, ncell, nt);
        NPC_LAUNCH(ctx);
        ctx->host_cache_keys[ntname] = key;
      }
      if (fwd_b0) {
        const int rb = 2 + nell;
        k_adj_b0_final<<<(nb + 127) / 128, 128, 0, ctx->stream>>>(sums, nt, nb, job.i33, ncell / ncell_s, ncell,
                                                                  job.out + (size_t)rb * nb,
                                                                  job.out + (size_t)(rb + 1) * nb);
        NPC_LAUNCH(ctx);
      }
    }
  }

  if (!job.grad) return NPC_OK;

  // 4. adjoint: B_0 term into Y, then (Y + 2 K X)/W back to the mesh
  C* Y = nullptr;
  if (job.dldb) {
    double* cb;
    NPC_TRY(ws_get(ctx, "adj.cb", sizeof(double) * nb, (void**)&cb));
    k_adj_bcoef<<<(nb + 127) / 128, 128, 0, ctx->stream>>>(nt, job.dldb, nb, job.i33, ncell / ncell_s, cb);
    NPC_LAUNCH(ctx);
    NPC_TRY(ws_get(ctx, "adj.Y", sizeof(C) * nrows * N, (void**)&Y));
    AFieldTable ft{};
    ft.nf = 0;
    for (int b = 0; b < nb; ++b) ft.f[ft.nf++] = AField{SRC_BIN, (int16_t)b, bin_radius(m.box, kb, b, KM), 0, 0};
    GradArgs ga{};
    NPC_TRY(shell_dispatch<T>(ctx, NS, ft, "sq", KM, N, X, bintab, ga, m.assign, ZMODE_SQUARE_FWD, nullptr, cb, Y,
                              nullptr));
  }
  GradArgs ga{};
  ga.Y = Y;
  ga.coef = coef;
  ga.nell = nell;
  for (int e = 0; e < nell; ++e) ga.ell[e] = ells[e];
  ga.nb = nb;
  for (int a = 0; a < 3; ++a) ga.los[a] = gl.los[a];
  AFieldTable ft{};
  ft.nf = 1;
  ft.f[0] = AField{SRC_GRAD, -1, KM, 0, 0};
  NPC_TRY((shell_pass<T, N>(ctx, ft, "grad", KM, N, X, bintab, ga, m.assign, ZMODE_WRITE, nullptr, nullptr, nullptr,
                            (T*)job.grad)));
  return NPC_OK;
}

template <typename T>
npc_status mesh_dispatch(npc_ctx* ctx, const npc_mesh_spec& m, const npc_kbins& kb, int prec, const void* mesh,
                         const MeshJob& job) {
  switch (m.n) {
    case 16: return mesh_impl<T, 16>(ctx, m, kb, prec, mesh, job);
    case 32: return mesh_impl<T, 32>(ctx, m, kb, prec, mesh, job);
    case 64: return mesh_impl<T, 64>(ctx, m, kb, prec, mesh, job);
    case 128: return mesh_impl<T, 128>(ctx, m, kb, prec, mesh, job);
    case 256: return mesh_impl<T, 256>(ctx, m, kb, prec, mesh, job);
  }
  if constexpr (sizeof(T) == 4) {
    if (m.n == 512) return mesh_impl<T, 512>(ctx, m, kb, prec, mesh, job);
    if (m.n == 1024) return mesh_impl<T, 1024>(ctx, m, kb, prec, mesh, job);
  }
  return set_err(ctx, NPC_ERR_UNSUPPORTED, "mesh size %d not supported at this precision", m.n);
}

int count_ells(uint32_t mask) { return (int)((mask & 1) + ((mask >> 2) & 1) + ((mask >> 4) & 1)); }

npc_status check_mesh_call(npc_ctx* ctx, const npc_mesh_spec* m, const npc_kbins* b, const void* mesh,
                           uint32_t ell_mask, int32_t b0, npc_precision prec) {
  NPC_TRY(check_spec(ctx, m));
  NPC_TRY(check_bins(ctx, b));
  if (m->n & (m->n - 1)) return set_err(ctx, NPC_ERR_UNSUPPORTED, "mesh estimators: n must be a power of two");
  if (!mesh) return set_err(ctx, NPC_ERR_INVALID_ARG, "mesh is NULL");
  if (!m->periodic || m->los != 1 || m->interlace != 0)
    return set_err(ctx, NPC_ERR_UNSUPPORTED, "mesh estimators: periodic box, global line of sight, no interlacing");
  if (ell_mask & ~0x15u) return set_err(ctx, NPC_ERR_INVALID_ARG, "ell_mask must use bits 0, 2, 4");
  if (b0 != 0 && b0 != 1) return set_err(ctx, NPC_ERR_INVALID_ARG, "b0 must be 0 or 1");
  if (ell_mask == 0 && b0 == 0) return set_err(ctx, NPC_ERR_INVALID_ARG, "nothing requested");
  if (prec != NPC_PREC_FP64 && prec != NPC_PREC_MIXED) return set_err(ctx, NPC_ERR_INVALID_ARG, "bad precision");
  if (prec == NPC_PREC_FP64 && m->n > 256) return set_err(ctx, NPC_ERR_UNSUPPORTED, "FP64 precision supports n <= 256");
  if (b0) {
    if (b->nbins > ADJ_MAX_FIELDS / 2) return set_err(ctx, NPC_ERR_UNSUPPORTED, "B_0 supports at most 32 bins");
    const double kf = 2.0 * M_PI / m->box;
    const double kmax = b->kmin + b->nbins * b->dk;
    if (kmax > 0.25 * kf * m->n)
      return set_err(ctx, NPC_ERR_UNSUPPORTED, "largest bin edge %.4g exceeds k_N/2 = %.4g", kmax, 0.25 * kf * m->n);
  }
  return NPC_OK;
}

}  // namespace

extern "C" {

int64_t npc_mesh_multipoles_len(const npc_kbins* bins, uint32_t ell_mask, int32_t b0) {
  if (!bins || bins->nbins < 1 || (ell_mask & ~0x15u) || (b0 != 0 && b0 != 1) || (ell_mask == 0 && !b0)) return 0;
  return (int64_t)(2 + count_ells(ell_mask) + 2 * b0) * bins->nbins;
}

npc_status npc_mesh_multipoles(npc_ctx* ctx, const npc_mesh_spec* spec, const void* mesh, const npc_kbins* bins,
                               uint32_t ell_mask, int32_t b0, double i22, double n0, double i33, npc_precision prec,
                               double* out, int32_t out_on_device) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  begin_call(ctx);
  NPC_TRY(check_mesh_call(ctx, spec, bins, mesh, ell_mask, b0, prec));
  if (!out) return set_err(ctx, NPC_ERR_INVALID_ARG, "out is NULL");
  if ((ell_mask && !(i22 > 0 && std::isfinite(i22))) || (b0 && !(i33 > 0 && std::isfinite(i33))) || !std::isfinite(n0))
    return set_err(ctx, NPC_ERR_NUMERIC, "normalisations must be finite and > 0");
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t len = npc_mesh_multipoles_len(bins, ell_mask, b0);
  double* dev_out = out;
  if (!out_on_device) NPC_TRY(ws_get(ctx, "adj.out", sizeof(double) * len, (void**)&dev_out));
  NPC_CUDA(ctx, cudaMemsetAsync(dev_out, 0, sizeof(double) * len, ctx->stream));
  MeshJob job{};
  job.n = spec->n;
  job.ell_mask = (int)ell_mask;
  job.want_b0 = b0;
  job.want_out = 1;
  job.i22 = i22;
  job.n0 = n0;
  job.i33 = i33;
  job.out = dev_out;
  ctx->stats.n_transforms = 1;
  ctx->stats.n_r2c_equivalent = 1;
  ctx->stats.n_phases = 1;
  NPC_TRY(stage_mark(ctx, "setup"));
  if (prec == NPC_PREC_FP64) NPC_TRY(mesh_dispatch<double>(ctx, *spec, *bins, prec, mesh, job));
  else NPC_TRY(mesh_dispatch<float>(ctx, *spec, *bins, prec, mesh, job));
  NPC_TRY(finish_output(ctx, dev_out, out, len, out_on_device));
  NPC_TRY(stage_mark(ctx, "download"));
  return end_call(ctx);
}

npc_status npc_mesh_multipoles_vjp(npc_ctx* ctx, const npc_mesh_spec* spec, const void* mesh, const npc_kbins* bins,
                                   uint32_t ell_mask, int32_t b0, double i22, double i33, const double* dl_dp,
                                   const double* dl_db0, int32_t cotangents_on_device, npc_precision prec,
                                   void* grad_mesh) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  begin_call(ctx);
  NPC_TRY(check_mesh_call(ctx, spec, bins, mesh, ell_mask, b0, prec));
  if (!grad_mesh) return set_err(ctx, NPC_ERR_INVALID_ARG, "grad_mesh is NULL");
  if (ell_mask && !dl_dp) return set_err(ctx, NPC_ERR_INVALID_ARG, "dl_dp is NULL while ell_mask != 0");
  if (b0 && !dl_db0) return set_err(ctx, NPC_ERR_INVALID_ARG, "dl_db0 is NULL while b0 = 1");
  if ((ell_mask && !(i22 > 0 && std::isfinite(i22))) || (b0 && !(i33 > 0 && std::isfinite(i33))))
    return set_err(ctx, NPC_ERR_NUMERIC, "normalisations must be finite and > 0");
  if (cotangents_on_device != 0 && cotangents_on_device != 1)
    return set_err(ctx, NPC_ERR_INVALID_ARG, "cotangents_on_device must be 0 or 1");
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));
  const int nb = bins->nbins;
  const int nell = count_ells(ell_mask);
  const double* dp = dl_dp;
  const double* db = dl_db0;
  if (!cotangents_on_device) {
    double* buf;
    NPC_TRY(ws_get(ctx, "adj.cot", sizeof(double) * (nell + 1) * nb, (void**)&buf));
    if (nell) {
      NPC_CUDA(ctx, cudaMemcpyAsync(buf, dl_dp, sizeof(double) * nell * nb, cudaMemcpyHostToDevice, ctx->stream));
      dp = buf;
    }
    if (b0) {
      NPC_CUDA(ctx, cudaMemcpyAsync(buf + (size_t)nell * nb, dl_db0, sizeof(double) * nb, cudaMemcpyHostToDevice,
                                    ctx->stream));
      db = buf + (size_t)nell * nb;
    }
  }
  MeshJob job{};
  job.n = spec->n;
  job.ell_mask = (int)ell_mask;
  job.want_b0 = b0;
  job.want_out = 0;
  job.i22 = i22;
  job.i33 = i33;
  job.dldp = nell ? dp : nullptr;
  job.dldb = b0 ? db : nullptr;
  job.grad = grad_mesh;
  ctx->stats.n_transforms = 1;
  ctx->stats.n_r2c_equivalent = 1;
  ctx->stats.n_phases = 1;
  NPC_TRY(stage_mark(ctx, "setup"));
  if (prec == NPC_PREC_FP64) NPC_TRY(mesh_dispatch<double>(ctx, *spec, *bins, prec, mesh, job));
  else NPC_TRY(mesh_dispatch<float>(ctx, *spec, *bins, prec, mesh, job));
  if (!cotangents_on_device) NPC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return end_call(ctx);
}

npc_status npc_paint_mesh(npc_ctx* ctx, const npc_mesh_spec* spec, const npc_catalog* data, npc_precision prec,
                          void* mesh) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  begin_call(ctx);
  NPC_TRY(check_spec(ctx, spec));
  NPC_TRY(check_catalog(ctx, data, "data", false));
  if (!mesh) return set_err(ctx, NPC_ERR_INVALID_ARG, "mesh is NULL");
  if (!spec->periodic || spec->interlace != 0)
    return set_err(ctx, NPC_ERR_UNSUPPORTED, "npc_paint_mesh: periodic box without interlacing");
  if (prec != NPC_PREC_FP64 && prec != NPC_PREC_MIXED) return set_err(ctx, NPC_ERR_INVALID_ARG, "bad precision");
  if (prec == NPC_PREC_FP64 && spec->n > 256) return set_err(ctx, NPC_ERR_UNSUPPORTED, "FP64 precision supports n <= 256");
  if (data->n == 0) return set_err(ctx, NPC_ERR_NUMERIC, "empty catalogue");
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));
  DevCatalog d;
  NPC_TRY(stage_catalog(ctx, data, "data", &d));
  double* sc;
  NPC_TRY(ws_get(ctx, "scalars", sizeof(double) * SC_COUNT, (void**)&sc));
  NPC_TRY(launch_catalog_scalars(ctx, d, nullptr, spec->box, sc));
  NPC_TRY(stage_mark(ctx, "scalars"));
  NPC_TRY(launch_paint(ctx, d, nullptr, *spec, 1, prec, sc, mesh, nullptr));
  NPC_TRY(stage_mark(ctx, "paint_fold"));
  return end_call(ctx);
}

npc_status npc_paint_adjoint(npc_ctx* ctx, const npc_mesh_spec* spec, const npc_catalog* data, const void* grad_mesh,
                             npc_precision prec, void* grad_pos, void* grad_w) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  begin_call(ctx);
  NPC_TRY(check_spec(ctx, spec));
  NPC_TRY(check_catalog(ctx, data, "data", false));
  if (!data->on_device && data->n > 0) return set_err(ctx, NPC_ERR_INVALID_ARG, "npc_paint_adjoint: device catalogue only");
  if (!grad_mesh || (!grad_pos && data->n > 0)) return set_err(ctx, NPC_ERR_INVALID_ARG, "grad_mesh / grad_pos is NULL");
  if (spec->interlace != 0) return set_err(ctx, NPC_ERR_UNSUPPORTED, "npc_paint_adjoint: one mesh (no interlacing)");
  if (prec != NPC_PREC_FP64 && prec != NPC_PREC_MIXED) return set_err(ctx, NPC_ERR_INVALID_ARG, "bad precision");
  if (prec == NPC_PREC_FP64 && spec->n > 256) return set_err(ctx, NPC_ERR_UNSUPPORTED, "FP64 precision supports n <= 256");
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));
  if (data->n == 0) return end_call(ctx);
  const int64_t np = data->n;
  const int grid = (int)std::min<int64_t>((np + 255) / 256, (int64_t)ctx->num_sms * 16);
  const double inv_h = (double)spec->n / spec->box;
  const double* o = spec->origin;
#define NPC_PADJ(A, TP, TG)                                                                                       \
  k_paint_adjoint<A, TP, TG><<<grid, 256, 0, ctx->stream>>>((const TP*)data->pos, (const TP*)data->w, np, spec->n, \
                                                            o[0], o[1], o[2], inv_h, (const TG*)grad_mesh,        \
                                                            (TP*)grad_pos, (TP*)grad_w)
  const bool p64 = data->dtype == 1, g64 = prec == NPC_PREC_FP64;
  if (spec->assign == 3) {
    if (p64 && g64) NPC_PADJ(3, double, double);
    else if (p64) NPC_PADJ(3, double, float);
    else if (g64) NPC_PADJ(3, float, double);
    else NPC_PADJ(3, float, float);
  } else {
    if (p64 && g64) NPC_PADJ(2, double, double);
    else if (p64) NPC_PADJ(2, double, float);
    else if (g64) NPC_PADJ(2, float, double);
    else NPC_PADJ(2, float, float);
  }
#undef NPC_PADJ
  NPC_LAUNCH(ctx);
  NPC_TRY(stage_mark(ctx, "paint_adjoint"));
  return end_call(ctx);
}

// Single-purpose forms of the calls above (float32 meshes, device memory)
npc_status npc_power_vjp(npc_ctx* ctx, const float* delta, const npc_mesh_spec* spec, const npc_kbins* bins,
                         uint32_t ell_mask, double i22, const double* dl_dp, float* dl_ddelta) {
  return npc_mesh_multipoles_vjp(ctx, spec, delta, bins, ell_mask, 0, i22, 1.0, dl_dp, nullptr, 0,
                                 NPC_PREC_MIXED, dl_ddelta);
}

npc_status npc_bispec0_vjp(npc_ctx* ctx, const float* delta, const npc_mesh_spec* spec, const npc_kbins* bins,
                           double i33, const double* dl_db0, float* dl_ddelta) {
  return npc_mesh_multipoles_vjp(ctx, spec, delta, bins, 0, 1, 1.0, i33, nullptr, dl_db0, 0, NPC_PREC_MIXED,
                                 dl_ddelta);
}

npc_status npc_tsc_adjoint(npc_ctx* ctx, const npc_mesh_spec* spec, const npc_catalog* data, const float* grad_mesh,
                           void* grad_pos) {
  if (spec && spec->assign != 3) {
    if (ctx) begin_call(ctx);
    return ctx ? set_err(ctx, NPC_ERR_INVALID_ARG, "npc_tsc_adjoint needs spec->assign = 3 (TSC)")
               : NPC_ERR_INVALID_ARG;
  }
  return npc_paint_adjoint(ctx, spec, data, grad_mesh, NPC_PREC_MIXED, grad_pos, nullptr);
}

}  // extern "C"
