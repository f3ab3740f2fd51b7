// Yamamoto power-spectrum multipoles from the m >= 0 spherical-harmonic weighted transforms.
//
// Each S_l^m(k) = sum_x F(x) Y_l^m(xhat) e^{-ik.x} with m >= 0 (Eq. key1) is the transform of the
// complex field F Y_l^m = F ReY + i F ImY; we transform its two real parts, A = FFT[F ReY] and
// B = FFT[F ImY], so S_l^m = A + iB and, by the conjugation symmetry the paper exploits (Eq.
// F_lm_SIC), S_l^{-m}(k) = (-1)^m [A(k) - iB(k)].  Summing over m (Eq. hand) then gives, with
// real coefficients only,
//   F_l(k) = 4 pi/(2l+1) [ Y_l0(khat) A_l0 + 2 sum_{m>=1} (ReY_lm(khat) A_lm + ImY_lm(khat) B_lm) ],
// which is Hermitian for even l: F_l is the space-inverted 1/2[G_l(k) + G_l^*(-k)] of Eq.
// F_and_new_G obtained directly, and Re<F_0 G_l^*> = <F_0 F_l^*> (Eq. pk_final).  All fields are
// real, so only the half spectrum kz in [0, n/2) is computed and stored (Nyquist planes are
// excluded from every bin) and every stored mode also stands for -k.
//
// Passes (3D transform by axes, shared-memory Stockham stages):
//   k_fwd_z           reads the painted meshes, applies Y_l^m(xhat) at each grid point (phase a
//                     at origin + jH, phase b at origin + (j - 1/2)H), transforms two real fields
//                     at a time as one complex column along z, splits them into two half spectra.
//   k_fft_cols        plain column transform along y.
//   k_fft_x_contract  transforms every field's x-row of one (ky, kz), then per mode: interlacing
//                     1/2[A_a + e^{iH(kx+ky+kz)/2} A_b], division by W(k) (Eq. compensation), F_l
//                     assembly, Re[F_0 F_l^*] and Re[F_l F_l'^*] (Eq. Pllp), binned in float64
//                     with a warp-segmented reduction into per-warp partial sums (no atomics
//                     between warps, fixed order: reproducible run to run).
//   k_power_finalize  fixed-order sum of the partials, normalisation (2l+1)/I22, shot noise,
//                     the modified multipoles of Eq. Plnew.
#include <cmath>

#include "fft_core.cuh"

namespace {

constexpr int CONTRACT_THREADS = 256;
constexpr int MAX_SUMS = 10;

template <int N> struct ColCfg {
  static constexpr int TX = N >= 1024 ? 4 : (N >= 512 ? 8 : 16);  // TX <= N
  static constexpr int THREADS = TX * N / 8;
};

// Weight of one real field at grid point (x, y, z): F times ReY/ImY of the direction from the
// observer to the grid point (phase b sits half a cell lower), or F alone (PART_ONE).
template <typename T>
struct ColGeom {
  T px[2], py[2], oz[2], h;   // per phase: x and y coordinates of this column, z origin
};

template <typename T>
__device__ __forceinline__ T comp_value(const Comp cp, const T* tileA, const T* tileB, int z, int c, int tx,
                                        const ColGeom<T>& cg, const YNorm& nrm) {
  if (cp.part == PART_ZERO) return T(0);
  const T F = (cp.phase ? tileB : tileA)[z * tx + c];
  if (cp.part == PART_ONE) return F;
  const int ph = cp.phase;
  const T pz = cg.oz[ph] + T(z) * cg.h;
  const T r2 = cg.px[ph] * cg.px[ph] + cg.py[ph] * cg.py[ph] + pz * pz;
  const T inv = r2 > T(0) ? rsqrt(r2) : T(0);
  T re, im;
  ylm_fast<T>(cp.ell, cp.m, cg.px[ph] * inv, cg.py[ph] * inv, pz * inv, nrm, re, im);
  return F * (cp.part == PART_RE ? re : im);
}

// First pass: weighted real fields -> half spectra along z.  Output layout half[f][kz][y][x].
template <typename T, int N>
__global__ void __launch_bounds__(ColCfg<N>::THREADS)
k_fwd_z(const T* __restrict__ mesh_a, const T* __restrict__ mesh_b, cplx<T>* __restrict__ half,
        const FieldList fl, const Geom g, const YNorm nrm, const cplx<T>* __restrict__ tw_g, int KZ) {
  using C = cplx<T>;
  constexpr int TX = ColCfg<N>::TX;
  constexpr int TPF = N / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* work = tw + N;
  T* tileA = reinterpret_cast<T*>(work + N * TX);
  T* tileB = tileA + N * TX;
  const int tid = threadIdx.x;
  const int c = tid % TX, t = tid / TX;
  const int x0 = blockIdx.x * TX, y = blockIdx.y;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = tw_g[i];
  for (int i = tid; i < N * TX; i += blockDim.x) {
    const int z = i / TX, cc = i % TX;
    const size_t gi = ((size_t)z * N + y) * N + x0 + cc;
    tileA[i] = mesh_a[gi];
    if (mesh_b) tileB[i] = mesh_b[gi];
  }
  ColGeom<T> cg;
  cg.h = (T)g.h;
  for (int ph = 0; ph < 2; ++ph) {
    const double sh = ph ? 0.5 : 0.0;
    cg.px[ph] = (T)(g.o[0] + ((double)(x0 + c) - sh) * g.h);
    cg.py[ph] = (T)(g.o[1] + ((double)y - sh) * g.h);
    cg.oz[ph] = (T)(g.o[2] - sh * g.h);
  }
  __syncthreads();
  const int npairs = (fl.nf + 1) / 2;
  const size_t fstride = (size_t)KZ * N * N;
  for (int p = 0; p < npairs; ++p) {
    const Comp c0 = fl.f[2 * p];
    Comp c1;
    c1.phase = 0; c1.ell = 0; c1.m = 0; c1.part = PART_ZERO;
    if (2 * p + 1 < fl.nf) c1 = fl.f[2 * p + 1];
    C v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int z = t + q * TPF;
      const T re = comp_value<T>(c0, tileA, tileB, z, c, TX, cg, nrm);
      const T im = comp_value<T>(c1, tileA, tileB, z, c, TX, cg, nrm);
      v[q] = cmk(re, im);
    }
    fft_block<N, -1>(v, t, tw, ColView<C>{work + c, TX});
#pragma unroll
    for (int q = 0; q < 8; ++q) work[(t + q * TPF) * TX + c] = v[q];
    __syncthreads();
    for (int i = tid; i < KZ * TX; i += blockDim.x) {
      const int kz = i / TX, cc = i % TX;
      const C z1 = work[kz * TX + cc];
      const C z2 = cconj(work[((N - kz) % N) * TX + cc]);
      const C a = cscale(cadd(z1, z2), T(0.5));
      const C d = csub(z1, z2);
      const C b = cmk(T(0.5) * d.y, T(-0.5) * d.x);
      const size_t gi = ((size_t)kz * N + y) * N + x0 + cc;
      half[(size_t)(2 * p) * fstride + gi] = a;
      if (2 * p + 1 < fl.nf) half[(size_t)(2 * p + 1) * fstride + gi] = b;
    }
    __syncthreads();
  }
}

// First pass for a single unweighted real field (global line of sight without interlacing, mesh
// gradients): two neighbouring x columns share one complex transform, c = F(x) + i F(x+1), and
// their half spectra follow from c(kz) and conj c(N - kz).  grid = (N / (2 TX), N).
template <int N> struct SingleCfg {   // column pairs per CTA: 2 TX divides N, TX <= the z-pass TX
  static constexpr int TX = (ColCfg<N>::TX >= 16 && N % 32 == 0) ? 16
                          : (ColCfg<N>::TX >= 8 && N % 16 == 0) ? 8 : 4;
  static constexpr int THREADS = TX * N / 8;
};

template <typename T, int N>
__global__ void __launch_bounds__(SingleCfg<N>::THREADS)
k_fwd_z_single(const T* __restrict__ mesh, cplx<T>* __restrict__ half, const cplx<T>* __restrict__ tw_g, int KZ) {
  using C = cplx<T>;
  constexpr int TX = SingleCfg<N>::TX;
  constexpr int TPF = N / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* work = tw + N;
  const int tid = threadIdx.x;
  const int c = tid % TX, t = tid / TX;
  const int x0 = blockIdx.x * 2 * TX, y = blockIdx.y;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = tw_g[i];
  C v[8];
  const T* col = mesh + (size_t)y * N + x0 + 2 * c;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const size_t zoff = (size_t)(t + q * TPF) * N * N;
    v[q] = cmk(col[zoff], col[zoff + 1]);
  }
  __syncthreads();
  fft_block<N, -1>(v, t, tw, ColView<C>{work + c, TX});
#pragma unroll
  for (int q = 0; q < 8; ++q) work[(t + q * TPF) * TX + c] = v[q];
  __syncthreads();
  for (int i = tid; i < KZ * TX; i += blockDim.x) {
    const int kz = i / TX, cc = i % TX;
    const C z1 = work[kz * TX + cc];
    const C z2 = cconj(work[((N - kz) % N) * TX + cc]);
    const C a = cscale(cadd(z1, z2), T(0.5));
    const C d = csub(z1, z2);
    const C b = cmk(T(0.5) * d.y, T(-0.5) * d.x);
    C* dst = half + ((size_t)kz * N + y) * N + x0 + 2 * cc;
    dst[0] = a;
    dst[1] = b;
  }
}

// ---------------------------------------------------------------------------------------------
// Specialised first pass for the standard interlaced field layout (l in {0, 2, 4}, both phases):
// pair p is (l, m, kind) known at compile time; kind 0 packs the m = 0 field of phase a (real
// part) with that of phase b (imaginary part), kind 1/2 is the complex field F Y_l^m of phase
// a/b whose real and imaginary parts share one Y evaluation.  Pairs are a prefix of
//   (0,0,0) (2,0,0) (2,1,1) (2,1,2) (2,2,1) (2,2,2) (4,0,0) (4,1,1) (4,1,2) ... (4,4,1) (4,4,2).
// ---------------------------------------------------------------------------------------------
// Polynomial factor Q_lm(uz) of Y_lm = norm_lm Q_lm(uz) (ux + i uy)^m, l <= 4: the associated
// Legendre function with its (-1)^m phase, divided by sin^m(theta).
template <typename T, int L, int M>
__device__ __forceinline__ T ylm_q(T uz) {
  const T z2 = uz * uz;
  if constexpr (L == 0) return T(1);
  else if constexpr (L == 1 && M == 0) return uz;
  else if constexpr (L == 1 && M == 1) return T(-1);
  else if constexpr (L == 3 && M == 0) return T(0.5) * uz * (T(5) * z2 - T(3));
  else if constexpr (L == 3 && M == 1) return T(-1.5) * (T(5) * z2 - T(1));
  else if constexpr (L == 3 && M == 2) return T(15) * uz;
  else if constexpr (L == 3 && M == 3) return T(-15);
  else if constexpr (L == 2 && M == 0) return T(1.5) * z2 - T(0.5);
  else if constexpr (L == 2 && M == 1) return T(-3) * uz;
  else if constexpr (L == 2 && M == 2) return T(3);
  else if constexpr (L == 4 && M == 0) return (T(35) * z2 * z2 - T(30) * z2 + T(3)) * T(0.125);
  else if constexpr (L == 4 && M == 1) return T(-2.5) * uz * (T(7) * z2 - T(3));
  else if constexpr (L == 4 && M == 2) return T(7.5) * (T(7) * z2 - T(1));
  else if constexpr (L == 4 && M == 3) return T(-105) * uz;
  else return T(105);
}

template <typename T, int L, int M>
__device__ __forceinline__ void ylm_ct(T ux, T uy, T uz, const YNorm& nrm, T& re, T& im) {
  const T q = ylm_q<T, L, M>(uz);
  T pr = T(1), pi = T(0);
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const T nr = pr * ux - pi * uy;
    pi = pr * uy + pi * ux;
    pr = nr;
  }
  const T c = ynorm<T>(nrm, L * (L + 1) / 2 + M) * q;
  re = c * pr;
  im = c * pi;
}

template <typename T> struct ZGeom {
  T px[2], py[2], pxy2[2];  // column x, row y per phase and px^2 + py^2
  T pz0[2];                 // z coordinate of element q = 0 of this thread, per phase
  T dz;                     // z step between consecutive elements of a thread (TPF cells)
};

// Keeps a value where it is computed: the per-pair factors below must not be hoisted out of the
// pair loop (all fifteen pairs' factors would then stay live in registers).
__device__ __forceinline__ void keep_here(float& x) { asm volatile("" : "+f"(x)); }
__device__ __forceinline__ void keep_here(double& x) { asm volatile("" : "+d"(x)); }

template <typename T, int N, int TX, int L, int M, int KIND>
__device__ __forceinline__ void std_inputs(cplx<T> (&v)[8], const T* tileA, const T* tileB, int c, int t,
                                           const ZGeom<T>& zg, const YNorm& nrm) {
  constexpr int TPF = N / 8;
  if constexpr (KIND == 0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int z = t + q * TPF;
      const T fa = tileA[z * TX + c], fb = tileB[z * TX + c];
      if constexpr (L == 0) {
        v[q] = cmk(fa, fb);
      } else {
        T ya, yb, dum;
        {
          const T pz = zg.pz0[0] + T(q) * zg.dz;
          const T inv = rsqrt(zg.pxy2[0] + pz * pz);
          ylm_ct<T, L, M>(zg.px[0] * inv, zg.py[0] * inv, pz * inv, nrm, ya, dum);
        }
        {
          const T pz = zg.pz0[1] + T(q) * zg.dz;
          const T inv = rsqrt(zg.pxy2[1] + pz * pz);
          ylm_ct<T, L, M>(zg.px[1] * inv, zg.py[1] * inv, pz * inv, nrm, yb, dum);
        }
        v[q] = cmk(fa * ya, fb * yb);
      }
    }
  } else {
    // Y_lm(xhat) = norm Q(uz) (px + i py)^m / r^m: the column factor norm (px + i py)^m is formed
    // once per pair, each element needs 1/r, uz and the power r^-m
    constexpr int ph = KIND - 1;
    T cr = ynorm<T>(nrm, L * (L + 1) / 2 + M), ci = T(0);
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const T nr = cr * zg.px[ph] - ci * zg.py[ph];
      ci = cr * zg.py[ph] + ci * zg.px[ph];
      cr = nr;
    }
    keep_here(cr);
    keep_here(ci);
    const T* tile = ph ? tileB : tileA;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int z = t + q * TPF;
      const T pz = zg.pz0[ph] + T(q) * zg.dz;
      const T inv = rsqrt(zg.pxy2[ph] + pz * pz);
      T s = tile[z * TX + c] * ylm_q<T, L, M>(pz * inv);
#pragma unroll
      for (int j = 0; j < M; ++j) s *= inv;
      v[q] = cmk(s * cr, s * ci);
    }
  }
}

// The real column signal of the (L, M > 0) fields of mesh phase PH: Y_LM(xhat) = norm Q_LM(uz)
// ((px + i py)/r)^M splits into s(z) = mesh(z) Q_LM(uz) r^-M, real, and the column factor
// cr + i ci = norm (px + i py)^M, constant along z; the transforms of the fields' real and imaginary
// parts are cr S(kz) and ci S(kz), S the transform of s.
template <typename T, int N, int TX, int L, int M, int PH>
__device__ __forceinline__ void std_real(T (&sv)[8], T& cr, T& ci, const T* tile, int c, int t, const ZGeom<T>& zg,
                                         const YNorm& nrm) {
  constexpr int TPF = N / 8;
  cr = ynorm<T>(nrm, L * (L + 1) / 2 + M);
  ci = T(0);
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const T nr = cr * zg.px[PH] - ci * zg.py[PH];
    ci = cr * zg.py[PH] + ci * zg.px[PH];
    cr = nr;
  }
  keep_here(cr);
  keep_here(ci);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int z = t + q * TPF;
    const T pz = zg.pz0[PH] + T(q) * zg.dz;
    const T inv = rsqrt(zg.pxy2[PH] + pz * pz);
    T v = tile[z * TX + c] * ylm_q<T, L, M>(pz * inv);
#pragma unroll
    for (int j = 0; j < M; ++j) v *= inv;
    sv[q] = v;
  }
}

// Phases a and b of one (L, M > 0): s_a + i s_b in one complex transform (two real signals), then
// S_a(k) = (Z(k) + Z(N - k)^*) / 2 and S_b(k) = (Z(k) - Z(N - k)^*) / 2i give the four half spectra.
template <typename T, int N, int TX, int L, int M>
__device__ __forceinline__ void std_pair_ab(cplx<T> (&v)[8], T (&cf)[4], const T* tileA, const T* tileB, int c, int t,
                                            const ZGeom<T>& zg, const YNorm& nrm) {
  T sa[8], sb[8];
  std_real<T, N, TX, L, M, 0>(sa, cf[0], cf[1], tileA, c, t, zg, nrm);
  std_real<T, N, TX, L, M, 1>(sb, cf[2], cf[3], tileB, c, t, zg, nrm);
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = cmk(sa[q], sb[q]);
}

// float: the occupancy of the form without packed phase pairs (64 registers at 512 threads, at most
// 80 otherwise), so that the pairs' extra live values do not cost CTAs per SM
template <typename T, int N> constexpr int zstd_min_blocks() {
  return sizeof(T) == 4 ? 65536 / (ColCfg<N>::THREADS * (ColCfg<N>::THREADS == 512 ? 64 : 80)) : 1;
}
template <typename T, int N>
__global__ void __launch_bounds__(ColCfg<N>::THREADS, zstd_min_blocks<T, N>())
k_fwd_z_std(const T* __restrict__ mesh_a, const T* __restrict__ mesh_b, cplx<T>* __restrict__ half, int npairs,
            const Geom g, const YNorm nrm, const cplx<T>* __restrict__ tw_g, int KZ) {
  using C = cplx<T>;
  constexpr int TX = ColCfg<N>::TX;
  constexpr int TPF = N / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* work = tw + N;
  T* tileA = reinterpret_cast<T*>(work + N * TX);
  T* tileB = tileA + N * TX;
  const int tid = threadIdx.x;
  const int c = tid % TX, t = tid / TX;
  const int x0 = blockIdx.x * TX, y = blockIdx.y;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = tw_g[i];
  for (int i = tid; i < N * TX; i += blockDim.x) {
    const int z = i / TX, cc = i % TX;
    const size_t gi = ((size_t)z * N + y) * N + x0 + cc;
    tileA[i] = mesh_a[gi];
    tileB[i] = mesh_b[gi];
  }
  ZGeom<T> zg;
  for (int ph = 0; ph < 2; ++ph) {
    const double sh = ph ? 0.5 : 0.0;
    zg.px[ph] = (T)(g.o[0] + ((double)(x0 + c) - sh) * g.h);
    zg.py[ph] = (T)(g.o[1] + ((double)y - sh) * g.h);
    zg.pxy2[ph] = zg.px[ph] * zg.px[ph] + zg.py[ph] * zg.py[ph];
    zg.pz0[ph] = (T)(g.o[2] + ((double)t - sh) * g.h);
  }
  zg.dz = (T)(g.h * TPF);
  __syncthreads();
  const size_t fstride = (size_t)KZ * N * N;
  for (int p = 0; p < npairs; ++p) {
    C v[8];
    // pairs 2k and 2k + 1 of an m > 0 harmonic (phase a, phase b): one transform for both
    const bool ab = (p == 2 || p == 4 || p == 7 || p == 9 || p == 11 || p == 13) && p + 1 < npairs;
    if (ab) {
      T cf[4];   // cr, ci of phase a, then of phase b
      switch (p) {
        case 2: std_pair_ab<T, N, TX, 2, 1>(v, cf, tileA, tileB, c, t, zg, nrm); break;
        case 4: std_pair_ab<T, N, TX, 2, 2>(v, cf, tileA, tileB, c, t, zg, nrm); break;
        case 7: std_pair_ab<T, N, TX, 4, 1>(v, cf, tileA, tileB, c, t, zg, nrm); break;
        case 9: std_pair_ab<T, N, TX, 4, 2>(v, cf, tileA, tileB, c, t, zg, nrm); break;
        case 11: std_pair_ab<T, N, TX, 4, 3>(v, cf, tileA, tileB, c, t, zg, nrm); break;
        default: std_pair_ab<T, N, TX, 4, 4>(v, cf, tileA, tileB, c, t, zg, nrm); break;
      }
      fft_block<N, -1>(v, t, tw, ColView<C>{work + c, TX});
#pragma unroll
      for (int q = 0; q < 8; ++q) work[(t + q * TPF) * TX + c] = v[q];
      __syncthreads();
      {
        // thread tid owns (kz0 + j KZSTEP, cc) with cc = tid % TX = c: its column's factors
        constexpr int KZSTEP = ColCfg<N>::THREADS / TX;
        const int kz0 = tid / TX, cc = tid % TX;
        C* o0 = half + (size_t)(2 * p) * fstride + ((size_t)kz0 * N + y) * N + x0 + cc;
        for (int kz = kz0; kz < KZ; kz += KZSTEP, o0 += (size_t)KZSTEP * N * N) {
          const C z1 = work[kz * TX + cc];
          const C z2 = cconj(work[(kz == 0 ? 0 : N - kz) * TX + cc]);
          const C sa = cscale(cadd(z1, z2), T(0.5));
          const C d = csub(z1, z2);
          const C sb = cmk(T(0.5) * d.y, T(-0.5) * d.x);
          o0[0] = cscale(sa, cf[0]);
          o0[fstride] = cscale(sa, cf[1]);
          o0[2 * fstride] = cscale(sb, cf[2]);
          o0[3 * fstride] = cscale(sb, cf[3]);
        }
      }
      __syncthreads();
      ++p;
      continue;
    }
    switch (p) {
      case 0: std_inputs<T, N, TX, 0, 0, 0>(v, tileA, tileB, c, t, zg, nrm); break;
      case 1: std_inputs<T, N, TX, 2, 0, 0>(v, tileA, tileB, c, t, zg, nrm); break;
      case 2: std_inputs<T, N, TX, 2, 1, 1>(v, tileA, tileB, c, t, zg, nrm); break;
      case 3: std_inputs<T, N, TX, 2, 1, 2>(v, tileA, tileB, c, t, zg, nrm); break;
      case 4: std_inputs<T, N, TX, 2, 2, 1>(v, tileA, tileB, c, t, zg, nrm); break;
      case 5: std_inputs<T, N, TX, 2, 2, 2>(v, tileA, tileB, c, t, zg, nrm); break;
      case 6: std_inputs<T, N, TX, 4, 0, 0>(v, tileA, tileB, c, t, zg, nrm); break;
      case 7: std_inputs<T, N, TX, 4, 1, 1>(v, tileA, tileB, c, t, zg, nrm); break;
      case 8: std_inputs<T, N, TX, 4, 1, 2>(v, tileA, tileB, c, t, zg, nrm); break;
      case 9: std_inputs<T, N, TX, 4, 2, 1>(v, tileA, tileB, c, t, zg, nrm); break;
      case 10: std_inputs<T, N, TX, 4, 2, 2>(v, tileA, tileB, c, t, zg, nrm); break;
      case 11: std_inputs<T, N, TX, 4, 3, 1>(v, tileA, tileB, c, t, zg, nrm); break;
      case 12: std_inputs<T, N, TX, 4, 3, 2>(v, tileA, tileB, c, t, zg, nrm); break;
      case 13: std_inputs<T, N, TX, 4, 4, 1>(v, tileA, tileB, c, t, zg, nrm); break;
      default: std_inputs<T, N, TX, 4, 4, 2>(v, tileA, tileB, c, t, zg, nrm); break;
    }
    fft_block<N, -1>(v, t, tw, ColView<C>{work + c, TX});
#pragma unroll
    for (int q = 0; q < 8; ++q) work[(t + q * TPF) * TX + c] = v[q];
    __syncthreads();
    // split the packed pair into its two half spectra; thread tid owns (kz0 + j KZSTEP, cc)
    {
      constexpr int KZSTEP = ColCfg<N>::THREADS / TX;
      const int kz0 = tid / TX, cc = tid % TX;
      C* o0 = half + (size_t)(2 * p) * fstride + ((size_t)kz0 * N + y) * N + x0 + cc;
      C* o1 = o0 + fstride;
      for (int kz = kz0; kz < KZ; kz += KZSTEP, o0 += (size_t)KZSTEP * N * N, o1 += (size_t)KZSTEP * N * N) {
        const C z1 = work[kz * TX + cc];
        const C z2 = cconj(work[(kz == 0 ? 0 : N - kz) * TX + cc]);
        *o0 = cscale(cadd(z1, z2), T(0.5));
        const C d = csub(z1, z2);
        *o1 = cmk(T(0.5) * d.y, T(-0.5) * d.x);
      }
    }
    __syncthreads();
  }
}

// Number of leading standard pairs the field list matches (0 if it does not follow the layout).
static int std_pairs(const FieldList& fl) {
  static const int8_t tbl[15][3] = {{0, 0, 0}, {2, 0, 0}, {2, 1, 1}, {2, 1, 2}, {2, 2, 1}, {2, 2, 2}, {4, 0, 0},
                                    {4, 1, 1}, {4, 1, 2}, {4, 2, 1}, {4, 2, 2}, {4, 3, 1}, {4, 3, 2}, {4, 4, 1},
                                    {4, 4, 2}};
  if (fl.nf % 2) return 0;
  const int np = fl.nf / 2;
  if (np > 15) return 0;
  for (int p = 0; p < np; ++p) {
    const Comp a = fl.f[2 * p], b = fl.f[2 * p + 1];
    const int l = tbl[p][0], m = tbl[p][1], kind = tbl[p][2];
    if (a.ell != l || b.ell != l || a.m != m || b.m != m) return 0;
    if (kind == 0) {
      const int part = l == 0 ? PART_ONE : PART_RE;
      if (a.phase != 0 || b.phase != 1 || a.part != part || b.part != part) return 0;
    } else {
      const int ph = kind - 1;
      if (a.phase != ph || b.phase != ph || a.part != PART_RE || b.part != PART_IM) return 0;
    }
  }
  return np;
}

// Column transform along a strided axis: element j of column (plane, x) at
// data[plane*plane_stride + j*row_stride + x].  grid = (N/TX, nplanes); TX columns per CTA is a
// tuning parameter (see tune_y_pass).
template <typename T, int N, int DIR, int TX>
__global__ void __launch_bounds__(TX * N / 8, (TX * N / 8 <= 512 ? 1536 / (TX * N / 8) : 1))
k_fft_cols(cplx<T>* __restrict__ data, size_t plane_stride, int row_stride, const cplx<T>* __restrict__ tw_g,
           int plane0, int kz_planes, int row_n2max) {
  using C = cplx<T>;
  constexpr int TPF = N / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* work = tw + N;
  const int tid = threadIdx.x;
  const int c = tid % TX, t = tid / TX;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = tw_g[i];
  C* base = data + (size_t)blockIdx.y * plane_stride + blockIdx.x * TX + c;
  C v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = base[(size_t)(t + q * TPF) * row_stride];
  __syncthreads();
  fft_block<N, DIR>(v, t, tw, ColView<C>{work + c, TX});
  // rows (ky, kz) outside every k-bin are never read again: not stored (plane p holds kz = p % kz_planes)
  const int kz = (plane0 + (int)blockIdx.y) % kz_planes;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int yi = t + q * TPF;
    const int jy = yi < N / 2 ? yi : yi - N;
    if (jy * jy + kz * kz <= row_n2max) base[(size_t)yi * row_stride] = v[q];
  }
}

// Per stored real field: which F_l it feeds, its mesh phase and its k-space coefficient
// scale * (ReY or ImY)(khat) from the row's Y table (scale = 4 pi/(2l+1) * (m > 0 ? 2 : 1)).
struct FieldCoef {
  int8_t acc;    // 0, 1, 2 for F_0, F_2, F_4
  int8_t phase;  // 0 or 1
  int8_t yidx;   // row Y-table index, -1 for PART_ONE
  int8_t part;   // PART_RE / PART_IM / PART_ONE
  float scale_f;
  double scale_d;
};
template <typename T> __device__ __forceinline__ T coef_scale(const FieldCoef& c);
template <> __device__ __forceinline__ float coef_scale<float>(const FieldCoef& c) { return c.scale_f; }
template <> __device__ __forceinline__ double coef_scale<double>(const FieldCoef& c) { return c.scale_d; }

// Row Y table: Y_lm(khat) in the fixed order (2,0) (2,1) (2,2) (4,0) .. (4,4) (1,0) (1,1) (3,0) .. (3,3).
constexpr int MAX_YTAB = 14;
__host__ __device__ constexpr int ytab_index(int l, int m) {
  return l == 2 ? m : (l == 4 ? 3 + m : (l == 1 ? 8 + m : 10 + m));
}
// Field slots of the x pass: slot[r * G + g] is the field row group g transforms in round r.
constexpr int MAX_SLOTS = 256;

struct ContractParams {
  int nf;
  FieldCoef fc[NPC_MAX_FIELDS];
  int ny;                       // Y table rows: 0, 3 (l = 2) or 8 (l = 2 and 4)
  int nacc;                     // F accumulators: nacc_b of F_0, F_2, F_4, then F_0^A if cross
  int nacc_b;
  int acc_a;                    // accumulator of F_0^A (cross spectra), -1 otherwise
  int nphase;
  int nrounds;                  // rounds of G field rows
  int phase_pure;               // 1: every group sees one mesh phase only (group parity when nphase = 2)
  int8_t slot[MAX_SLOTS];       // field per (round, group), -1 for none
  int nbins, nsum;
  int row_n2max;                // rows (ky, kz) with ky^2 + kz^2 above this hold no binned mode
  int KZ;                       // planes kz < KZ stored per field by the forward passes
  int nell;
  int ell_list[5];
  int nll;
  int lla[3], llb[3];
  int need2, need4;
  int need_mask;                // multipoles l whose F_l the binning forms (bit l)
  int acc_of[5];                // accumulator of F_l (tracer B), -1 if none
  int ymask;                    // Y table groups evaluated per row: bit l for l = 1 .. 4
  int even_layout;              // acc_of = {0, -1, 1 or -1, -1, 2 or -1}: the fixed even-l layout
  int global_los;
  double los[3];
  int assign;
  double kf;
};

template <typename T>
__device__ __forceinline__ T sinc_pow(T a, int p) {
  const T s = a == T(0) ? T(1) : sin(a) / a;
  T r = s;
  for (int i = 1; i < p; ++i) r *= s;
  return r;
}

__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }

template <int N> struct XCfg {
  static constexpr int TPF = N / 8;
  static constexpr int G = RowGroups<N, CONTRACT_THREADS>::G;        // rows in flight
  static constexpr int NBUF = RowGroups<N, CONTRACT_THREADS>::NBUF;  // exchange buffers
};

// Last pass.  For one (ky, kz) row: every field row is transformed along x and added, with its
// coefficient, into per-group F_l accumulators (F_l is linear in the fields, so the 30 rows never
// need to be resident together); then per mode the products Re[F_0 F_l^*], Re[F_l F_l'^*] are
// binned.  Groups own their accumulators and threads own their modes, so no shared-memory
// atomics are needed, and the group sum runs in a fixed order.
template <typename T, int N>
__global__ void __launch_bounds__(CONTRACT_THREADS, 2)
k_fft_x_contract(const cplx<T>* __restrict__ half, const ContractParams P, const YNorm nrm,
                 const int16_t* __restrict__ bintab, const cplx<T>* __restrict__ tw_g, double* __restrict__ part) {
  using C = cplx<T>;
  constexpr int TPF = XCfg<N>::TPF;
  constexpr int G = XCfg<N>::G;
  constexpr int NP = row_pad_len<N>();
  constexpr int NW = CONTRACT_THREADS / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* ytab = tw + N;                         // [ny][N]
  C* facc = ytab + (size_t)P.ny * N;        // [G][nacc][N]
  C* rowbuf = facc + (size_t)G * P.nacc * N;  // [G][NP]
  C* fb = rowbuf + (size_t)XCfg<N>::NBUF * NP;  // phase-b factor per kx: fa e^{i pi (i+j+l)/N}
  T* winv = reinterpret_cast<T*>(fb + N);   // 1/sinc^p, a = 0..N/2
  T* fa = winv + (N / 2 + 2);               // phase-a factor per kx
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = tw_g[i];
  for (int i = tid; i <= N / 2; i += blockDim.x) winv[i] = T(1) / sinc_pow<T>(T(M_PI) * T(i) / T(N), P.assign);
  __syncthreads();
  double* mypart = part + ((size_t)blockIdx.x * NW + warp) * P.nbins * P.nsum;
  const int nrows = P.KZ * N;
  const int g = tid / TPF, t = tid % TPF;
  const bool ingroup = g < G;
  const T half_or_one = P.nphase == 2 ? T(0.5) : T(1);
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int kz = r / N, ky = r % N;
    const int jy = ky < N / 2 ? ky : ky - N;
    if (jy * jy + kz * kz > P.row_n2max) continue;   // block-uniform: the whole row is outside the bins
    // per-mode window/interlace factor and Y_lm(khat) table; clear the accumulators
    for (int kx = tid; kx < N; kx += blockDim.x) {
      const int i = kx < N / 2 ? kx : kx - N;
      const int ai = i < 0 ? -i : i, aj = jy < 0 ? -jy : jy;
      fa[kx] = half_or_one * winv[ai] * winv[aj] * winv[kz];
      {
        // interlacing phase e^{i pi (i + j + l)/N}, the argument reduced to (-1, 1] half turns
        int m = i + jy + kz;
        m = ((m % (2 * N)) + 2 * N) % (2 * N);
        if (m > N) m -= 2 * N;
        T sn, cs;
        sincospi_t(T(m) / T(N), &sn, &cs);
        fb[kx] = cmk(cs * fa[kx], sn * fa[kx]);
      }
      if (P.ny > 0) {
        const T fi = T(i), fj = T(jy), fk = T(kz);
        const T r2 = fi * fi + fj * fj + fk * fk;
        const T inv = r2 > T(0) ? rsqrt(r2) : T(0);
        const T ux = fi * inv, uy = fj * inv, uz = r2 > T(0) ? fk * inv : T(1);
        T re, im;
        if (P.ymask & 2) {
          ylm_ct<T, 1, 0>(ux, uy, uz, nrm, re, im); ytab[8 * N + kx] = cmk(re, im);
          ylm_ct<T, 1, 1>(ux, uy, uz, nrm, re, im); ytab[9 * N + kx] = cmk(re, im);
        }
        if (P.ymask & 8) {
          ylm_ct<T, 3, 0>(ux, uy, uz, nrm, re, im); ytab[10 * N + kx] = cmk(re, im);
          ylm_ct<T, 3, 1>(ux, uy, uz, nrm, re, im); ytab[11 * N + kx] = cmk(re, im);
          ylm_ct<T, 3, 2>(ux, uy, uz, nrm, re, im); ytab[12 * N + kx] = cmk(re, im);
          ylm_ct<T, 3, 3>(ux, uy, uz, nrm, re, im); ytab[13 * N + kx] = cmk(re, im);
        }
        ylm_ct<T, 2, 0>(ux, uy, uz, nrm, re, im); ytab[0 * N + kx] = cmk(re, im);
        ylm_ct<T, 2, 1>(ux, uy, uz, nrm, re, im); ytab[1 * N + kx] = cmk(re, im);
        ylm_ct<T, 2, 2>(ux, uy, uz, nrm, re, im); ytab[2 * N + kx] = cmk(re, im);
        if (P.ymask & 16) {
          ylm_ct<T, 4, 0>(ux, uy, uz, nrm, re, im); ytab[3 * N + kx] = cmk(re, im);
          ylm_ct<T, 4, 1>(ux, uy, uz, nrm, re, im); ytab[4 * N + kx] = cmk(re, im);
          ylm_ct<T, 4, 2>(ux, uy, uz, nrm, re, im); ytab[5 * N + kx] = cmk(re, im);
          ylm_ct<T, 4, 3>(ux, uy, uz, nrm, re, im); ytab[6 * N + kx] = cmk(re, im);
          ylm_ct<T, 4, 4>(ux, uy, uz, nrm, re, im); ytab[7 * N + kx] = cmk(re, im);
        }
      }
      for (int q = 0; q < G * P.nacc; ++q) facc[(size_t)q * N + kx] = cmk(T(0), T(0));
    }
    __syncthreads();
    C v[8], vn[8], racc[8];
    int cur = -1;   // accumulator held in racc
    const size_t fstride = (size_t)P.KZ * N * N;
    const size_t roff = ((size_t)kz * N + ky) * N;
    int f = ingroup ? P.slot[g] : -1;
    if (f >= 0) {
      const C* src = half + (size_t)f * fstride + roff;
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = src[t + q * TPF];
    }
    for (int rd = 0; rd < P.nrounds; ++rd) {
      const bool live = f >= 0;
      const int fn = (ingroup && rd + 1 < P.nrounds) ? P.slot[(rd + 1) * G + g] : -1;
      if (fn >= 0) {
        const C* src = half + (size_t)fn * fstride + roff;
#pragma unroll
        for (int q = 0; q < 8; ++q) vn[q] = src[t + q * TPF];
      }
      if (!live) {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = cmk(T(0), T(0));
      }
      fft_block<N, -1>(v, t, tw, RowView<C>{rowbuf + (size_t)(ingroup ? g : G) * NP},
                       RowSync<N, CONTRACT_THREADS>::make(g));
      if (live) {
        const FieldCoef c = P.fc[f];
        if (c.acc != cur) {   // a group's fields come in accumulator order: flush once per change
          if (cur >= 0) {
            C* acc = facc + ((size_t)g * P.nacc + cur) * N;
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[t + q * TPF] = cadd(acc[t + q * TPF], racc[q]);
          }
          cur = c.acc;
#pragma unroll
          for (int q = 0; q < 8; ++q) racc[q] = cmk(T(0), T(0));
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int kx = t + q * TPF;
          T w = coef_scale<T>(c);
          if (c.yidx >= 0) {
            const C y = ytab[(size_t)c.yidx * N + kx];
            w *= (c.part == PART_RE ? y.x : y.y);
          }
          // phase-pure groups apply the window and interlacing factors once per mode, at binning
          const C a = P.phase_pure ? cscale(v[q], w)
                                   : (c.phase ? cmul(v[q], cscale(fb[kx], w)) : cscale(v[q], w * fa[kx]));
          racc[q] = cadd(racc[q], a);
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = vn[q];
      f = fn;
    }
    if (cur >= 0) {
      C* acc = facc + ((size_t)g * P.nacc + cur) * N;
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[t + q * TPF] = cadd(acc[t + q * TPF], racc[q]);
    }
    __syncthreads();
    const T fjy = T(jy), fkz = T(kz);
    // modes kx = jp and kx = -jp (index N - jp) have the same |k|, hence the same bin: where a thread
    // would bin two or more modes, it adds the mirror pair before the warp-segmented scan (one scan
    // and one set of run-end atomics per pair); smaller rows keep one mode per thread
    constexpr bool MIRROR = N >= 2 * CONTRACT_THREADS;
    constexpr int NJ = MIRROR ? N / 2 : N;
    for (int jb = warp * 32; jb < NJ; jb += blockDim.x) {
      const int jp = jb + lane;
      int bin = -1;
      T vals[MAX_SUMS];
#pragma unroll
      for (int s = 0; s < MAX_SUMS; ++s) vals[s] = T(0);
#pragma unroll 1
      for (int mir = 0; mir < (MIRROR ? 2 : 1); ++mir) {
        const int j = MIRROR ? (mir ? N - jp : jp) : jp;
        const int i = MIRROR ? (mir ? -jp : jp) : (jp < N / 2 ? jp : jp - N);
        const bool in_row = MIRROR ? (jp < N / 2 && (mir == 0 || jp > 0)) : (jp < N && i != -N / 2);
        int mbin = -1;
        if (in_row && jy != -N / 2 && (i != 0 || jy != 0 || kz != 0)) mbin = bintab[i * i + jy * jy + kz * kz];
        if (mbin >= 0) {
          bin = mbin;
          const T wgt = kz > 0 ? T(2) : T(1);
          // accumulators summed over the groups: phase a (even g, or all with one phase) and phase b
          C Aa[6], Ab[6];
#pragma unroll
          for (int a = 0; a < 6; ++a) Aa[a] = Ab[a] = cmk(T(0), T(0));
          auto gsum = [&](int g0, int gstep, C (&acc)[6]) {
            for (int gg = g0; gg < G; gg += gstep) {
              const C* fg = facc + (size_t)gg * P.nacc * N + j;
#pragma unroll
              for (int a = 0; a < 6; ++a)
                if (a < P.nacc) acc[a] = cadd(acc[a], fg[(size_t)a * N]);
            }
          };
          if (P.phase_pure) {
            gsum(0, P.nphase == 2 ? 2 : 1, Aa);
            const T faj = fa[j];
#pragma unroll
            for (int a = 0; a < 6; ++a) Aa[a] = cscale(Aa[a], faj);
            if (P.nphase == 2) {
              gsum(1, 2, Ab);
              const C fbj = fb[j];
#pragma unroll
              for (int a = 0; a < 6; ++a) Aa[a] = cadd(Aa[a], cmul(Ab[a], fbj));
            }
          } else {
            gsum(0, 1, Aa);
          }
          auto pick = [&](int k) {   // accumulator k (runtime index kept out of local memory)
            C r = cmk(T(0), T(0));
#pragma unroll
            for (int a = 0; a < 6; ++a)
              if (k == a) r = Aa[a];
            return r;
          };
          const C F0 = Aa[0];
          C F1, F2, F3, F4, FA;
          if (P.even_layout) {   // accumulators F_0, F_2, F_4 (when present) at 0, 1, 2, then F_0^A
            F1 = F3 = cmk(T(0), T(0));
            F2 = Aa[1];
            F4 = Aa[2];
            FA = P.acc_a == 1 ? Aa[1] : (P.acc_a == 2 ? Aa[2] : Aa[3]);
          } else {
            F1 = pick(P.acc_of[1]);
            F2 = pick(P.acc_of[2]);
            F3 = pick(P.acc_of[3]);
            F4 = pick(P.acc_of[4]);
            FA = pick(P.acc_a);
          }
          const T fi = T(i);
          const T kk = sqrt(fi * fi + fjy * fjy + fkz * fkz);
          if (P.global_los) {
            const T mu = (fi * T(P.los[0]) + fjy * T(P.los[1]) + fkz * T(P.los[2])) / kk;
            if (P.need_mask & 2) F1 = cscale(F0, legendre_p<T>(1, mu));
            if (P.need_mask & 4) F2 = cscale(F0, legendre_p<T>(2, mu));
            if (P.need_mask & 8) F3 = cscale(F0, legendre_p<T>(3, mu));
            if (P.need_mask & 16) F4 = cscale(F0, legendre_p<T>(4, mu));
          }
          auto sel = [&](int l) { return l == 0 ? F0 : (l == 1 ? F1 : (l == 2 ? F2 : (l == 3 ? F3 : F4))); };
#pragma unroll
          for (int s = 0; s < MAX_SUMS; ++s) {
            T v = T(0);
            if (s < P.nell) {
              const int l = P.ell_list[s];
              const C b = sel(l);
              const C a = P.acc_a >= 0 ? FA : F0;   // cross: F_0 of tracer A against F_l of B
              // even l: Re a b^*; odd l: Im a b^* (Sec. 2.1, odd multipoles)
              v = wgt * ((l & 1) ? (a.y * b.x - a.x * b.y) : (a.x * b.x + a.y * b.y));
            } else if (s < P.nell + P.nll) {
              const C a = sel(P.lla[s - P.nell]), b = sel(P.llb[s - P.nell]);
              v = wgt * (a.x * b.x + a.y * b.y);
            } else if (s == P.nsum - 2) {
              v = wgt;
            } else if (s == P.nsum - 1) {
              v = wgt * T(P.kf) * kk;
            }
            vals[s] += v;
          }
        }
      }
      // warp-segmented inclusive scan over runs of consecutive lanes with equal bin; a run is
      // identified by the number of run heads up to this lane, so runs of the same bin that are
      // not adjacent (a warp spanning both kx halves when n < 64) stay separate
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
      // run sums over at most 32 modes stay in T; only run ends convert to float64
#pragma unroll
      for (int s = 0; s < MAX_SUMS; ++s) {
        if (s >= P.nsum) break;
        T x = vals[s];
#pragma unroll
        for (int st = 0; st < 5; ++st) {
          const T yv = __shfl_up_sync(0xffffffffu, x, 1 << st);
          if (addm & (1u << st)) x += yv;
        }
        if (last && bin >= 0) atomicAdd(mypart + (size_t)bin * P.nsum + s, (double)x);
      }
    }
    __syncthreads();
  }
}

struct FinalParams {
  int nbins, nsum, nparts;
  int nell, ell_list[5];
  int nll, lla[3], llb[3];
  int nmod, mod_list[3];
  int out_rows;          // 2 + requested P_l + requested P_lb + requested P_ll'
  int ll_req;            // output P_22 (bit 0), P_42 (bit 1), P_44 (bit 2)
  int req_mask;          // requested P_l (bits)
};

constexpr int FIN_THREADS = 128;

// one block per bin: the partials are summed with a fixed per-thread stride and a fixed tree
__global__ void __launch_bounds__(FIN_THREADS)
k_power_finalize(const double* __restrict__ part, const FinalParams F, const double* __restrict__ sc,
                 double* __restrict__ out) {
  const int nb = F.nbins;
  __shared__ double red[MAX_SUMS][FIN_THREADS];
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    double S[MAX_SUMS];
    for (int s = 0; s < MAX_SUMS; ++s) S[s] = 0.0;
    for (int p = threadIdx.x; p < F.nparts; p += FIN_THREADS)
      for (int s = 0; s < F.nsum; ++s) S[s] += part[((size_t)p * nb + b) * F.nsum + s];
    for (int s = 0; s < MAX_SUMS; ++s) red[s][threadIdx.x] = S[s];
    __syncthreads();
    for (int off = FIN_THREADS / 2; off > 0; off >>= 1) {
      if (threadIdx.x < off)
        for (int s = 0; s < MAX_SUMS; ++s) red[s][threadIdx.x] += red[s][threadIdx.x + off];
      __syncthreads();
    }
    for (int s = 0; s < MAX_SUMS; ++s) S[s] = red[s][0];
    __syncthreads();
    if (threadIdx.x != 0) continue;
    const double cnt = S[F.nsum - 2];
    const double i22 = sc[SC_I22], n0 = sc[SC_N0];
    const bool ok = cnt > 0;
    out[0 * nb + b] = ok ? S[F.nsum - 1] / cnt : 0.0;
    out[1 * nb + b] = cnt;
    double Pl[5] = {0, 0, 0, 0, 0};   // index l
    int row = 2;
    for (int e = 0; e < F.nell; ++e) {
      const int l = F.ell_list[e];
      const double v = ok ? (2 * l + 1) / i22 * S[e] / cnt - (l == 0 ? n0 : 0.0) : 0.0;
      Pl[l] = v;
      if (F.req_mask & (1 << l)) out[(row++) * nb + b] = v;
    }
    double P22 = 0, P42 = 0, P44 = 0;
    for (int e = 0; e < F.nll; ++e) {
      const int a = F.lla[e], c = F.llb[e];
      const double nsh = (a == c) ? (2 * (a + c) + 1) * n0 / (2 * a + 1) : 0.0;
      const double v = ok ? (2 * (a + c) + 1) / i22 * S[F.nell + e] / cnt - nsh : 0.0;
      if (a == 2 && c == 2) P22 = v;
      if (a == 4 && c == 2) P42 = v;
      if (a == 4 && c == 4) P44 = v;
    }
    for (int e = 0; e < F.nmod; ++e) {
      const int lb = F.mod_list[e];
      double v = 0.0;
      if (ok) {
        if (lb == 4) v = 35.0 / 18.0 * P22 - Pl[2] - 3.5 * Pl[0];
        if (lb == 6) v = 11.0 / 5.0 * P42 - 52.0 / 63.0 * Pl[4] - 286.0 / 175.0 * Pl[2];
        if (lb == 8)
          v = 1287.0 / 490.0 * P44 - 374.0 / 245.0 * P42 - 3553.0 / 15435.0 * Pl[4] - 1326.0 / 8575.0 * Pl[2] -
              2431.0 / 490.0 * Pl[0];
      }
      out[(row++) * nb + b] = v;
    }
    // the two-index spectra themselves (Eq. Pllp), when requested: P_22, P_42, P_44
    if (F.ll_req & 1) out[(row++) * nb + b] = P22;
    if (F.ll_req & 2) out[(row++) * nb + b] = P42;
    if (F.ll_req & 4) out[(row++) * nb + b] = P44;
  }
  if (blockIdx.x == 0 && threadIdx.x < 8) out[(size_t)F.out_rows * nb + threadIdx.x] = sc[threadIdx.x];
}

// ---------------------------------------------------------------------------------------------
// y pass with a selectable number of columns per CTA
// ---------------------------------------------------------------------------------------------
template <int N> constexpr bool ytx_ok(int tx) { return tx <= N && N % tx == 0 && tx * N / 8 <= 1024; }

int ytx_for(const npc_ctx* ctx, int n, bool fp64) {
  auto it = ctx->ytx.find(n * 2 + (fp64 ? 1 : 0));
  if (it != ctx->ytx.end()) return it->second;
  return n >= 1024 ? 4 : (n >= 512 ? 8 : 16);
}

template <typename T, int N, int TX>
npc_status y_pass_tx(npc_ctx* ctx, cplx<T>* data, int nplanes, const cplx<T>* tw, int kz_planes, int row_n2max) {
  using C = cplx<T>;
  if constexpr (!ytx_ok<N>(TX)) {
    return set_err(ctx, NPC_ERR_INVALID_ARG, "y pass: %d columns per CTA not valid at n = %d", TX, N);
  } else {
    const size_t smem = sizeof(C) * (N + N * TX);
    auto kern = k_fft_cols<T, N, -1, TX>;
    NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int p0 = 0; p0 < nplanes; p0 += 65535) {
      const int np = std::min(65535, nplanes - p0);
      kern<<<dim3(N / TX, np), TX * N / 8, smem, ctx->stream>>>(data + (size_t)p0 * N * N, (size_t)N * N, N, tw, p0,
                                                                kz_planes, row_n2max);
      NPC_LAUNCH(ctx);
    }
    return NPC_OK;
  }
}

template <typename T, int N>
npc_status y_pass(npc_ctx* ctx, cplx<T>* data, int nplanes, const cplx<T>* tw, int tx, int kz_planes = 1,
                  int row_n2max = 1 << 30) {
  switch (tx) {
    case 4: return y_pass_tx<T, N, 4>(ctx, data, nplanes, tw, kz_planes, row_n2max);
    case 8: return y_pass_tx<T, N, 8>(ctx, data, nplanes, tw, kz_planes, row_n2max);
    case 16: return y_pass_tx<T, N, 16>(ctx, data, nplanes, tw, kz_planes, row_n2max);
    case 32: return y_pass_tx<T, N, 32>(ctx, data, nplanes, tw, kz_planes, row_n2max);
  }
  return set_err(ctx, NPC_ERR_INVALID_ARG, "y pass: unsupported columns per CTA %d", tx);
}

// Autotuner for the y pass: times every valid columns-per-CTA choice on a scratch buffer of
// `nplanes` planes (values irrelevant to the timing) and keeps the fastest for (n, precision).
template <typename T, int N>
npc_status tune_y_impl(npc_ctx* ctx, int nplanes) {
  using C = cplx<T>;
  const void* twp;
  NPC_TRY(get_twiddles(ctx, N, sizeof(T) == 8 ? NPC_PREC_FP64 : NPC_PREC_MIXED, &twp));
  C* buf;
  NPC_TRY(ws_get(ctx, "tune.y", sizeof(C) * (size_t)nplanes * N * N, (void**)&buf));
  NPC_CUDA(ctx, cudaMemsetAsync(buf, 0, sizeof(C) * (size_t)nplanes * N * N, ctx->stream));
  cudaEvent_t e0, e1;
  NPC_CUDA(ctx, cudaEventCreate(&e0));
  NPC_CUDA(ctx, cudaEventCreate(&e1));
  float best = 1e30f;
  int best_tx = ytx_for(ctx, N, sizeof(T) == 8);
  npc_status st = NPC_OK;
  for (int tx : {4, 8, 16, 32}) {
    if (!(tx <= N && N % tx == 0 && tx * N / 8 <= 1024)) continue;
    st = y_pass<T, N>(ctx, buf, nplanes, (const C*)twp, tx);  // warm-up
    if (st != NPC_OK) break;
    cudaEventRecord(e0, ctx->stream);
    for (int rep = 0; rep < 3 && st == NPC_OK; ++rep) st = y_pass<T, N>(ctx, buf, nplanes, (const C*)twp, tx);
    cudaEventRecord(e1, ctx->stream);
    if (st != NPC_OK) break;
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_tx = tx;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != NPC_OK) return st;
  ctx->ytx[N * 2 + (sizeof(T) == 8 ? 1 : 0)] = best_tx;
  return NPC_OK;
}

// ---------------------------------------------------------------------------------------------
template <typename T, int N>
npc_status fwd_impl(npc_ctx* ctx, const PowerPlan& plan, const Geom& g, const void* mesh_a, const void* mesh_b,
                    void* half) {
  const int KZ = plan.kz_keep > 0 ? std::min(plan.kz_keep, N / 2) : N / 2;
  using C = cplx<T>;
  constexpr int TX = ColCfg<N>::TX;
  const void* twp;
  NPC_TRY(get_twiddles(ctx, N, sizeof(T) == 8 ? NPC_PREC_FP64 : NPC_PREC_MIXED, &twp));
  const C* tw = (const C*)twp;
  const YNorm nrm = ylm_norm_table();
  {
    const size_t smem = sizeof(C) * (N + N * TX) + sizeof(T) * 2 * N * TX;
    dim3 grid(N / TX, N);
    const int nstd = mesh_b ? std_pairs(plan.fl) : 0;
    const bool single = !mesh_b && plan.fl.nf == 1 && plan.fl.f[0].part == PART_ONE && plan.fl.f[0].phase == 0;
    if (single) {
      constexpr int STX = SingleCfg<N>::TX;
      static_assert(N % (2 * STX) == 0, "column pairs must tile the mesh");
      const size_t ssmem = sizeof(C) * (N + N * STX);
      auto kern = k_fwd_z_single<T, N>;
      NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssmem));
      kern<<<dim3(N / (2 * STX), N), SingleCfg<N>::THREADS, ssmem, ctx->stream>>>((const T*)mesh_a, (C*)half, tw,
                                                                                   KZ);
    } else if (nstd > 0) {
      auto kern = k_fwd_z_std<T, N>;
      NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<grid, ColCfg<N>::THREADS, smem, ctx->stream>>>((const T*)mesh_a, (const T*)mesh_b, (C*)half, nstd, g,
                                                            nrm, tw, KZ);
    } else {
      auto kern = k_fwd_z<T, N>;
      NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<grid, ColCfg<N>::THREADS, smem, ctx->stream>>>((const T*)mesh_a, (const T*)mesh_b, (C*)half, plan.fl,
                                                            g, nrm, tw, KZ);
    }
    NPC_LAUNCH(ctx);
    NPC_TRY(stage_mark(ctx, "fft_z_weighted"));
  }
  // planes (f, kz) are contiguous N*N blocks; y rows have stride N
  NPC_TRY((y_pass<T, N>(ctx, (C*)half, plan.fl.nf * KZ, tw, ytx_for(ctx, N, sizeof(T) == 8), KZ,
                        plan.row_n2max > 0 ? plan.row_n2max : (1 << 30))));
  NPC_TRY(stage_mark(ctx, "fft_y"));
  return NPC_OK;
}

template <typename T, int N>
npc_status contract_impl(npc_ctx* ctx, const PowerPlan& plan, const npc_mesh_spec& m, const npc_kbins& kb,
                         const void* half, const double* sc, double* dev_out) {
  using C = cplx<T>;
  const void* twp;
  NPC_TRY(get_twiddles(ctx, N, sizeof(T) == 8 ? NPC_PREC_FP64 : NPC_PREC_MIXED, &twp));
  const int16_t* bintab;
  NPC_TRY(get_bin_table(ctx, N, m.box, kb, &bintab));
  ContractParams P{};
  P.nf = plan.fl.nf;
  P.nphase = plan.nphase;
  P.ny = 0;
  int req_internal = plan.ells_mask;
  if (plan.mod_mask) req_internal |= 1 | 4 | 16;
  P.need2 = (req_internal & 4) ? 1 : 0;
  P.need4 = (req_internal & 16) ? 1 : 0;
  P.need_mask = req_internal | 1;
  // accumulators: one per multipole with fields of tracer B (in l order), then F_0^A
  for (int l = 0; l <= 4; ++l) P.acc_of[l] = -1;
  P.nacc_b = 0;
  if (plan.global_los) {
    P.acc_of[0] = 0;
    P.nacc_b = 1;
  } else {
    for (int l = 0; l <= 4; ++l) {
      bool has = false;
      for (int f = 0; f < plan.fl.nf; ++f) has |= !plan.fl.f[f].tracer && plan.fl.f[f].ell == l;
      if (has) P.acc_of[l] = P.nacc_b++;
    }
  }
  P.acc_a = plan.cross ? P.nacc_b : -1;
  P.nacc = P.nacc_b + (plan.cross ? 1 : 0);
  if (P.nacc > 6) return set_err(ctx, NPC_ERR_UNSUPPORTED, "x pass: at most 6 accumulators");
  P.even_layout = (P.acc_of[1] < 0 && P.acc_of[3] < 0 && (P.acc_of[2] == 1 || P.acc_of[2] < 0) &&
                   (P.acc_of[4] == 2 || P.acc_of[4] < 0) && (P.acc_a < 0 || P.acc_a <= 3)) ? 1 : 0;
  if (plan.cross && plan.mod_mask)
    return set_err(ctx, NPC_ERR_UNSUPPORTED, "cross spectra: no modified multipoles");
  P.ymask = 0;
  for (int f = 0; f < plan.fl.nf; ++f) {
    const Comp c = plan.fl.f[f];
    FieldCoef fc;
    fc.acc = (int8_t)(c.tracer ? P.acc_a : (plan.global_los ? 0 : P.acc_of[c.ell]));
    if (c.tracer && (!plan.cross || c.part != PART_ONE))
      return set_err(ctx, NPC_ERR_INVALID_ARG, "x pass: tracer-A field must be an unweighted F_0");
    fc.phase = c.phase;
    fc.part = c.part;
    fc.yidx = -1;
    fc.scale_d = 1.0;
    fc.scale_f = 1.0f;
    if (c.part == PART_RE || c.part == PART_IM) {
      if (c.ell < 1 || c.ell > 4 || c.m < 0 || c.m > c.ell)
        return set_err(ctx, NPC_ERR_UNSUPPORTED, "Y_%d%d field in the x pass", c.ell, c.m);
      fc.yidx = (int8_t)ytab_index(c.ell, c.m);
      P.ymask |= 1 << c.ell;
      P.ny = std::max(P.ny, (P.ymask & 10) ? 14 : ((P.ymask & 16) ? 8 : 3));
      fc.scale_d = 4.0 * M_PI / (2 * c.ell + 1) * (c.m > 0 ? 2.0 : 1.0);
      fc.scale_f = (float)fc.scale_d;
    }
    P.fc[f] = fc;
  }
  {
    // field slots: with two phases and an even number of row groups, even groups take the
    // phase-a fields and odd groups the phase-b fields (in list order), so that a group's
    // accumulators hold one phase and the window/interlacing factors are applied per mode
    constexpr int G = XCfg<N>::G;
    std::vector<int> ph[2];
    for (int f = 0; f < plan.fl.nf; ++f) ph[plan.fl.f[f].phase ? 1 : 0].push_back(f);
    P.phase_pure = (P.nphase == 1 || G % 2 == 0) ? 1 : 0;
    if (P.nphase == 1 && !ph[1].empty()) return set_err(ctx, NPC_ERR_INVALID_ARG, "phase-b field without interlacing");
    int nrounds;
    if (P.phase_pure && P.nphase == 2) {
      const int per = G / 2;
      nrounds = (int)std::max((ph[0].size() + per - 1) / per, (ph[1].size() + per - 1) / per);
    } else {
      nrounds = (plan.fl.nf + G - 1) / G;
    }
    if ((size_t)nrounds * G > (size_t)MAX_SLOTS)
      return set_err(ctx, NPC_ERR_UNSUPPORTED, "x pass: %d fields do not fit %d slots", plan.fl.nf, MAX_SLOTS);
    P.nrounds = nrounds;
    for (int r = 0; r < nrounds; ++r)
      for (int g = 0; g < G; ++g) {
        int f = -1;
        if (P.phase_pure && P.nphase == 2) {
          const size_t i = (size_t)r * (G / 2) + g / 2;
          const std::vector<int>& l = ph[g & 1];
          if (i < l.size()) f = l[i];
        } else {
          const int i = r * G + g;
          if (i < plan.fl.nf) f = i;
        }
        P.slot[r * G + g] = (int8_t)f;
      }
  }
  P.nbins = kb.nbins;
  P.nell = 0;
  for (int l = 0; l <= 4; ++l)
    if (req_internal & (1 << l)) P.ell_list[P.nell++] = l;
  P.nll = 0;
  if (plan.mod_mask & ((1 << 4) | (1 << 16))) { P.lla[P.nll] = 2; P.llb[P.nll] = 2; P.nll++; }
  if (plan.mod_mask & ((1 << 6) | (1 << 8) | (1 << 17))) { P.lla[P.nll] = 4; P.llb[P.nll] = 2; P.nll++; }
  if (plan.mod_mask & ((1 << 8) | (1 << 18))) { P.lla[P.nll] = 4; P.llb[P.nll] = 4; P.nll++; }
  P.nsum = P.nell + P.nll + 2;
  P.KZ = plan.kz_keep > 0 ? std::min(plan.kz_keep, N / 2) : N / 2;
  P.global_los = plan.global_los;
  for (int a = 0; a < 3; ++a) P.los[a] = plan.los[a];
  P.assign = plan.assign;
  P.kf = 2.0 * M_PI / m.box;
  {
    // a mode is binned only if k_f |q| < kmin + nbins dk; its row has ky^2 + kz^2 <= |q|^2
    const double kmax = kb.kmin + kb.nbins * kb.dk;
    const double r2 = std::pow(kmax / P.kf, 2);
    P.row_n2max = r2 >= 3.0 * (N / 2) * (N / 2) ? 3 * (N / 2) * (N / 2) : (int)std::floor(r2) + 1;
  }

  constexpr int NP = row_pad_len<N>();
  constexpr int G = XCfg<N>::G;
  const size_t smem = sizeof(C) * ((size_t)N + (size_t)P.ny * N + (size_t)G * P.nacc * N +
                                   (size_t)XCfg<N>::NBUF * NP + N) +
                      sizeof(T) * (N / 2 + 2 + N);
  auto kern = k_fft_x_contract<T, N>;
  NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  NPC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CONTRACT_THREADS, smem));
  if (per_sm < 1) return set_err(ctx, NPC_ERR_UNSUPPORTED, "contraction does not fit on an SM (%zu B smem)", smem);
  const int nrows = P.KZ * N;
  const int grid = std::min(nrows, per_sm * ctx->num_sms);
  const int nw = CONTRACT_THREADS / 32;
  const size_t nparts = (size_t)grid * nw;
  double* part;
  NPC_TRY(ws_get(ctx, "power.part", sizeof(double) * nparts * P.nbins * P.nsum, (void**)&part));
  NPC_CUDA(ctx, cudaMemsetAsync(part, 0, sizeof(double) * nparts * P.nbins * P.nsum, ctx->stream));
  NPC_TRY(stage_mark(ctx, "contract_setup"));
  kern<<<grid, CONTRACT_THREADS, smem, ctx->stream>>>((const C*)half, P, ylm_norm_table(), bintab, (const C*)twp,
                                                      part);
  NPC_LAUNCH(ctx);
  NPC_TRY(stage_mark(ctx, "fft_x_contract"));

  FinalParams F{};
  F.nbins = P.nbins;
  F.nsum = P.nsum;
  F.nparts = (int)nparts;
  F.nell = P.nell;
  for (int e = 0; e < P.nell; ++e) F.ell_list[e] = P.ell_list[e];
  F.nll = P.nll;
  for (int e = 0; e < P.nll; ++e) { F.lla[e] = P.lla[e]; F.llb[e] = P.llb[e]; }
  F.nmod = 0;
  for (int lb = 4; lb <= 8; lb += 2)
    if (plan.mod_mask & (1 << lb)) F.mod_list[F.nmod++] = lb;
  int nreq = 0;
  for (int l = 0; l <= 4; ++l) nreq += (plan.ells_mask >> l) & 1;
  F.ll_req = (plan.mod_mask >> 16) & 7;
  F.out_rows = 2 + nreq + F.nmod + ((F.ll_req & 1) + ((F.ll_req >> 1) & 1) + ((F.ll_req >> 2) & 1));
  F.req_mask = plan.ells_mask;
  k_power_finalize<<<std::min(P.nbins, 1024), FIN_THREADS, 0, ctx->stream>>>(part, F, sc, dev_out);
  NPC_LAUNCH(ctx);
  NPC_TRY(stage_mark(ctx, "finalize"));
  return NPC_OK;
}

// float32 transforms for n = 2^k in [16, 1024] and n = 48, 96, 192; float64 transforms for n <= 256
template <typename T>
npc_status fwd_dispatch(npc_ctx* ctx, const PowerPlan& plan, const Geom& g, const void* a, const void* b, void* half) {
  switch (plan.n) {
    case 16: return fwd_impl<T, 16>(ctx, plan, g, a, b, half);
    case 32: return fwd_impl<T, 32>(ctx, plan, g, a, b, half);
    case 64: return fwd_impl<T, 64>(ctx, plan, g, a, b, half);
    case 128: return fwd_impl<T, 128>(ctx, plan, g, a, b, half);
    case 256: return fwd_impl<T, 256>(ctx, plan, g, a, b, half);
    case 48: return fwd_impl<T, 48>(ctx, plan, g, a, b, half);
    case 96: return fwd_impl<T, 96>(ctx, plan, g, a, b, half);
    case 192: return fwd_impl<T, 192>(ctx, plan, g, a, b, half);
  }
  if constexpr (sizeof(T) == 4) {
    if (plan.n == 512) return fwd_impl<T, 512>(ctx, plan, g, a, b, half);
    if (plan.n == 1024) return fwd_impl<T, 1024>(ctx, plan, g, a, b, half);
  }
  return set_err(ctx, NPC_ERR_UNSUPPORTED, "mesh size %d not supported at this precision", plan.n);
}

template <typename T>
npc_status contract_dispatch(npc_ctx* ctx, const PowerPlan& plan, const npc_mesh_spec& m, const npc_kbins& kb,
                             const void* half, const double* sc, double* out) {
  switch (plan.n) {
    case 16: return contract_impl<T, 16>(ctx, plan, m, kb, half, sc, out);
    case 32: return contract_impl<T, 32>(ctx, plan, m, kb, half, sc, out);
    case 64: return contract_impl<T, 64>(ctx, plan, m, kb, half, sc, out);
    case 128: return contract_impl<T, 128>(ctx, plan, m, kb, half, sc, out);
    case 256: return contract_impl<T, 256>(ctx, plan, m, kb, half, sc, out);
    case 48: return contract_impl<T, 48>(ctx, plan, m, kb, half, sc, out);
    case 96: return contract_impl<T, 96>(ctx, plan, m, kb, half, sc, out);
    case 192: return contract_impl<T, 192>(ctx, plan, m, kb, half, sc, out);
  }
  if constexpr (sizeof(T) == 4) {
    if (plan.n == 512) return contract_impl<T, 512>(ctx, plan, m, kb, half, sc, out);
    if (plan.n == 1024) return contract_impl<T, 1024>(ctx, plan, m, kb, half, sc, out);
  }
  return set_err(ctx, NPC_ERR_UNSUPPORTED, "mesh size %d not supported at this precision", plan.n);
}

}  // namespace

npc_status tune_y_pass(npc_ctx* ctx, int n, int prec, int nplanes) {
  const bool d = prec == NPC_PREC_FP64;
#define NPC_TY(NN)                                                              \
  case NN:                                                                      \
    return d ? tune_y_impl<double, NN>(ctx, nplanes) : tune_y_impl<float, NN>(ctx, nplanes);
  switch (n) {
    NPC_TY(16) NPC_TY(32) NPC_TY(48) NPC_TY(64) NPC_TY(96) NPC_TY(128) NPC_TY(192) NPC_TY(256)
    case 512: return d ? set_err(ctx, NPC_ERR_UNSUPPORTED, "FP64 n <= 256") : tune_y_impl<float, 512>(ctx, nplanes);
    case 1024: return d ? set_err(ctx, NPC_ERR_UNSUPPORTED, "FP64 n <= 256") : tune_y_impl<float, 1024>(ctx, nplanes);
  }
#undef NPC_TY
  return set_err(ctx, NPC_ERR_UNSUPPORTED, "mesh size %d", n);
}

npc_status run_forward_transforms(npc_ctx* ctx, int prec, const PowerPlan& plan, const Geom& g,
                                  const void* mesh_a, const void* mesh_b, void* half) {
  if (prec == NPC_PREC_FP64) {
    if (plan.n > 256) return set_err(ctx, NPC_ERR_UNSUPPORTED, "FP64 precision supports n <= 256");
    return fwd_dispatch<double>(ctx, plan, g, mesh_a, mesh_b, half);
  }
  return fwd_dispatch<float>(ctx, plan, g, mesh_a, mesh_b, half);
}

npc_status run_power_contract(npc_ctx* ctx, int prec, const PowerPlan& plan, const npc_mesh_spec& m,
                              const npc_kbins& kb, const void* half, const double* sc, double* dev_out) {
  if (prec == NPC_PREC_FP64) return contract_dispatch<double>(ctx, plan, m, kb, half, sc, dev_out);
  return contract_dispatch<float>(ctx, plan, m, kb, half, sc, dev_out);
}
