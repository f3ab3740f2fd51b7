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
constexpr int MAX_SUMS = 8;

template <int N> struct ColCfg {
  static constexpr int TX = N >= 1024 ? 4 : (N >= 512 ? 8 : 16);  // TX <= N
  static constexpr int THREADS = TX * N / 8;
};

template <typename T>
__device__ __forceinline__ T comp_value(const Comp cp, const T* tileA, const T* tileB, int z, int c,
                                        int tx, int x, int y, const Geom& g, const YNorm& nrm) {
  if (cp.part == PART_ZERO) return T(0);
  const T F = (cp.phase ? tileB : tileA)[z * tx + c];
  if (cp.part == PART_ONE) return F;
  const T sh = cp.phase ? T(0.5) : T(0);
  const T h = (T)g.h;
  const T px = (T)g.o[0] + (T(x) - sh) * h;
  const T py = (T)g.o[1] + (T(y) - sh) * h;
  const T pz = (T)g.o[2] + (T(z) - sh) * h;
  const T r2 = px * px + py * py + pz * pz;
  const T inv = r2 > T(0) ? T(1) / sqrt(r2) : T(0);
  T re, im;
  ylm_eval<T>(cp.ell, cp.m, px * inv, py * inv, pz * inv, nrm, re, im);
  return F * (cp.part == PART_RE ? re : im);
}

// First pass: weighted real fields -> half spectra along z.  Output layout half[f][kz][y][x].
template <typename T, int N>
__global__ void __launch_bounds__(ColCfg<N>::THREADS)
k_fwd_z(const T* __restrict__ mesh_a, const T* __restrict__ mesh_b, cplx<T>* __restrict__ half,
        const FieldList fl, const Geom g, const YNorm nrm, const cplx<T>* __restrict__ tw_g) {
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
  __syncthreads();
  const int npairs = (fl.nf + 1) / 2;
  const size_t fstride = (size_t)(N / 2) * N * N;
  for (int p = 0; p < npairs; ++p) {
    const Comp c0 = fl.f[2 * p];
    Comp c1;
    c1.phase = 0; c1.ell = 0; c1.m = 0; c1.part = PART_ZERO;
    if (2 * p + 1 < fl.nf) c1 = fl.f[2 * p + 1];
    C v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int z = t + q * TPF;
      const T re = comp_value<T>(c0, tileA, tileB, z, c, TX, x0 + c, y, g, nrm);
      const T im = comp_value<T>(c1, tileA, tileB, z, c, TX, x0 + c, y, g, nrm);
      v[q] = cmk(re, im);
    }
    fft_block<N, -1>(v, t, tw, ColView<C>{work + c, TX});
#pragma unroll
    for (int q = 0; q < 8; ++q) work[(t + q * TPF) * TX + c] = v[q];
    __syncthreads();
    for (int i = tid; i < (N / 2) * TX; i += blockDim.x) {
      const int kz = i / TX, cc = i % TX;
      const C z1 = work[kz * TX + cc];
      const C z2 = cconj(work[((N - kz) & (N - 1)) * TX + cc]);
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

// Column transform along a strided axis: element j of column (plane, x) at
// data[plane*plane_stride + j*row_stride + x].  grid = (N/TX, nplanes).
template <typename T, int N, int DIR>
__global__ void __launch_bounds__(ColCfg<N>::THREADS)
k_fft_cols(cplx<T>* __restrict__ data, size_t plane_stride, int row_stride, const cplx<T>* __restrict__ tw_g) {
  using C = cplx<T>;
  constexpr int TX = ColCfg<N>::TX;
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
#pragma unroll
  for (int q = 0; q < 8; ++q) base[(size_t)(t + q * TPF) * row_stride] = v[q];
}

struct LogicalField {   // one (l, m, part) with its field index per phase
  int8_t ell, m, part;
  int8_t idx0, idx1;    // idx1 = -1 without interlacing
};

struct ContractParams {
  int nf;               // stored real fields
  int nlog;             // logical fields
  LogicalField lf[NPC_MAX_FIELDS];
  int nphase;
  int nbins, nsum;
  int nell;             // P_l sums for ell_list
  int ell_list[3];
  int nll;              // two-index sums
  int lla[3], llb[3];
  int need2, need4;     // F_2, F_4 required
  int global_los;
  float los[3];
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

template <typename T, int N>
__global__ void __launch_bounds__(CONTRACT_THREADS)
k_fft_x_contract(const cplx<T>* __restrict__ half, const ContractParams P, const YNorm nrm,
                 const int16_t* __restrict__ bintab, const cplx<T>* __restrict__ tw_g, double* __restrict__ part) {
  using C = cplx<T>;
  constexpr int TPF = N / 8;
  constexpr int G = CONTRACT_THREADS / TPF > 0 ? CONTRACT_THREADS / TPF : 1;
  constexpr int NP = row_pad_len<N>();
  constexpr int NW = CONTRACT_THREADS / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* phs = tw + N;                 // e^{i pi a / N}, a = -N/2 .. N/2-1  (index a + N/2)
  T* winv = reinterpret_cast<T*>(phs + N);   // 1 / sinc(pi a/N)^p, a = 0 .. N/2
  C* rows = reinterpret_cast<C*>(winv + (N / 2 + 2));
  C* dummy = rows + (size_t)P.nf * NP;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < N; i += blockDim.x) {
    tw[i] = tw_g[i];
    const T a = T(M_PI) * T(i - N / 2) / T(N);
    phs[i] = cmk(cos(a), sin(a));
  }
  for (int i = tid; i <= N / 2; i += blockDim.x) winv[i] = T(1) / sinc_pow<T>(T(M_PI) * T(i) / T(N), P.assign);
  __syncthreads();
  double* mypart = part + ((size_t)blockIdx.x * NW + warp) * P.nbins * P.nsum;
  const int nrows = (N / 2) * N;
  const int g = tid / TPF, t = tid % TPF;
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int kz = r / N, ky = r % N;
    for (int f0 = 0; f0 < P.nf; f0 += G) {
      const int f = f0 + g;
      C v[8];
      const bool live = (g < G) && (f < P.nf);
      if (live) {
        const C* src = half + (((size_t)f * (N / 2) + kz) * N + ky) * N;
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = src[t + q * TPF];
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = cmk(T(0), T(0));
      }
      RowView<C> rv{live ? rows + (size_t)f * NP : dummy};
      fft_block<N, -1>(v, t, tw, rv);
      if (live) {
#pragma unroll
        for (int q = 0; q < 8; ++q) rv.st(t + q * TPF, v[q]);
      }
    }
    __syncthreads();
    const int jy = ky < N / 2 ? ky : ky - N;
    for (int jb = warp * 32; jb < N; jb += blockDim.x) {
      const int j = jb + lane;
      const int i = j < N / 2 ? j : j - N;
      int bin = -1;
      if (j < N && i != -N / 2 && jy != -N / 2 && (i != 0 || jy != 0 || kz != 0)) bin = bintab[i * i + jy * jy + kz * kz];
      double vals[MAX_SUMS];
#pragma unroll
      for (int s = 0; s < MAX_SUMS; ++s) vals[s] = 0.0;
      if (bin >= 0) {
        const T wgt = kz > 0 ? T(2) : T(1);
        const int ai = i < 0 ? -i : i, aj = jy < 0 ? -jy : jy;
        const T iw = winv[ai] * winv[aj] * winv[kz];
        C ph = cmk(T(1), T(0));
        if (P.nphase == 2) ph = cmul(cmul(phs[i + N / 2], phs[jy + N / 2]), phs[kz + N / 2]);
        const T kk = sqrt(T(i * i + jy * jy + kz * kz));
        const T ux = T(i) / kk, uy = T(jy) / kk, uz = T(kz) / kk;
        C F0 = cmk(T(0), T(0)), F2 = cmk(T(0), T(0)), F4 = cmk(T(0), T(0));
        const int jp = RowView<C>::idx(j);
        for (int k = 0; k < P.nlog; ++k) {
          const LogicalField L = P.lf[k];
          C a = rows[(size_t)L.idx0 * NP + jp];
          if (L.idx1 >= 0) a = cscale(cadd(a, cmul(ph, rows[(size_t)L.idx1 * NP + jp])), T(0.5));
          a = cscale(a, iw);
          T coef;
          if (L.part == PART_ONE) {
            coef = T(1);
          } else {
            T re, im;
            ylm_eval<T>(L.ell, L.m, ux, uy, uz, nrm, re, im);
            coef = T(4.0 * M_PI) / T(2 * L.ell + 1) * (L.m > 0 ? T(2) : T(1)) * (L.part == PART_RE ? re : im);
          }
          const C term = cscale(a, coef);
          if (L.ell == 0) F0 = cadd(F0, term);
          else if (L.ell == 2) F2 = cadd(F2, term);
          else F4 = cadd(F4, term);
        }
        if (P.global_los) {
          const T mu = ux * T(P.los[0]) + uy * T(P.los[1]) + uz * T(P.los[2]);
          if (P.need2) F2 = cscale(F0, legendre_p<T>(2, mu));
          if (P.need4) F4 = cscale(F0, legendre_p<T>(4, mu));
        }
        const C Fl[3] = {F0, F2, F4};
        int s = 0;
        for (int e = 0; e < P.nell; ++e, ++s) {
          const C b = Fl[P.ell_list[e] / 2];
          vals[s] = (double)(wgt * (F0.x * b.x + F0.y * b.y));
        }
        for (int e = 0; e < P.nll; ++e, ++s) {
          const C a = Fl[P.lla[e] / 2], b = Fl[P.llb[e] / 2];
          vals[s] = (double)(wgt * (a.x * b.x + a.y * b.y));
        }
        vals[P.nsum - 2] = (double)wgt;
        vals[P.nsum - 1] = (double)wgt * P.kf * (double)kk;
      }
      // warp-segmented inclusive scan over runs of equal bin (|k| is monotone along a warp of
      // consecutive kx within one half of the row, so equal bins are contiguous for n >= 64)
      unsigned addm = 0;
#pragma unroll
      for (int st = 0; st < 5; ++st) {
        const int off = 1 << st;
        const int ob = __shfl_up_sync(0xffffffffu, bin, off);
        if (lane >= off && ob == bin) addm |= 1u << st;
      }
      const int nb = __shfl_down_sync(0xffffffffu, bin, 1);
      const bool last = (lane == 31) || (nb != bin);
      for (int s = 0; s < P.nsum; ++s) {
        double x = vals[s];
#pragma unroll
        for (int st = 0; st < 5; ++st) {
          const double y = __shfl_up_sync(0xffffffffu, x, 1 << st);
          if (addm & (1u << st)) x += y;
        }
        if (last && bin >= 0) atomicAdd(mypart + (size_t)bin * P.nsum + s, x);
      }
    }
    __syncthreads();
  }
}

struct FinalParams {
  int nbins, nsum, nparts;
  int nell, ell_list[3];
  int nll, lla[3], llb[3];
  int nmod, mod_list[3];
  int out_rows;          // 2 + requested P_l + requested P_lb
  int req_mask;          // requested P_l (bits)
};

__global__ void k_power_finalize(const double* __restrict__ part, const FinalParams F, const double* __restrict__ sc,
                                 double* __restrict__ out) {
  const int nb = F.nbins;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    double S[MAX_SUMS];
    for (int s = 0; s < F.nsum; ++s) S[s] = 0.0;
    for (int p = 0; p < F.nparts; ++p)
      for (int s = 0; s < F.nsum; ++s) S[s] += part[((size_t)p * nb + b) * F.nsum + s];
    const double cnt = S[F.nsum - 2];
    const double i22 = sc[SC_I22], n0 = sc[SC_N0];
    const bool ok = cnt > 0;
    out[0 * nb + b] = ok ? S[F.nsum - 1] / cnt : 0.0;
    out[1 * nb + b] = cnt;
    double Pl[5] = {0, 0, 0, 0, 0};   // index l/2
    int row = 2;
    for (int e = 0; e < F.nell; ++e) {
      const int l = F.ell_list[e];
      const double v = ok ? (2 * l + 1) / i22 * S[e] / cnt - (l == 0 ? n0 : 0.0) : 0.0;
      Pl[l / 2] = v;
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
        if (lb == 4) v = 35.0 / 18.0 * P22 - Pl[1] - 3.5 * Pl[0];
        if (lb == 6) v = 11.0 / 5.0 * P42 - 52.0 / 63.0 * Pl[2] - 286.0 / 175.0 * Pl[1];
        if (lb == 8)
          v = 1287.0 / 490.0 * P44 - 374.0 / 245.0 * P42 - 3553.0 / 15435.0 * Pl[2] - 1326.0 / 8575.0 * Pl[1] -
              2431.0 / 490.0 * Pl[0];
      }
      out[(row++) * nb + b] = v;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < 8) out[(size_t)F.out_rows * nb + threadIdx.x] = sc[threadIdx.x];
}

// ---------------------------------------------------------------------------------------------
template <typename T, int N>
npc_status fwd_impl(npc_ctx* ctx, const PowerPlan& plan, const Geom& g, const void* mesh_a, const void* mesh_b,
                    void* half) {
  using C = cplx<T>;
  constexpr int TX = ColCfg<N>::TX;
  const void* twp;
  NPC_TRY(get_twiddles(ctx, N, sizeof(T) == 8 ? NPC_PREC_FP64 : NPC_PREC_MIXED, &twp));
  const C* tw = (const C*)twp;
  const YNorm nrm = ylm_norm_table();
  {
    const size_t smem = sizeof(C) * (N + N * TX) + sizeof(T) * 2 * N * TX;
    auto kern = k_fwd_z<T, N>;
    NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(N / TX, N);
    kern<<<grid, ColCfg<N>::THREADS, smem, ctx->stream>>>((const T*)mesh_a, (const T*)mesh_b, (C*)half, plan.fl, g,
                                                          nrm, tw);
    NPC_LAUNCH(ctx);
  }
  {
    const size_t smem = sizeof(C) * (N + N * TX);
    auto kern = k_fft_cols<T, N, -1>;
    NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int nplanes = plan.fl.nf * (N / 2);
    // planes (f, kz) are contiguous N*N blocks; y rows have stride N
    for (int p0 = 0; p0 < nplanes; p0 += 65535) {
      const int np = std::min(65535, nplanes - p0);
      dim3 grid(N / TX, np);
      kern<<<grid, ColCfg<N>::THREADS, smem, ctx->stream>>>((C*)half + (size_t)p0 * N * N, (size_t)N * N, N, tw);
      NPC_LAUNCH(ctx);
    }
  }
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
  // logical fields: pair up the per-phase copies of each (l, m, part)
  P.nlog = 0;
  for (int f = 0; f < plan.fl.nf; ++f) {
    const Comp c = plan.fl.f[f];
    if (c.phase != 0 || c.part == PART_ZERO) continue;
    LogicalField L;
    L.ell = c.ell; L.m = c.m; L.part = c.part; L.idx0 = (int8_t)f; L.idx1 = -1;
    for (int f2 = 0; f2 < plan.fl.nf; ++f2) {
      const Comp d = plan.fl.f[f2];
      if (d.phase == 1 && d.ell == c.ell && d.m == c.m && d.part == c.part) L.idx1 = (int8_t)f2;
    }
    P.lf[P.nlog++] = L;
  }
  P.nbins = kb.nbins;
  P.nell = 0;
  int req_internal = plan.ells_mask;
  if (plan.mod_mask) req_internal |= 1 | 4 | 16;
  for (int l = 0; l <= 4; l += 2)
    if (req_internal & (1 << l)) P.ell_list[P.nell++] = l;
  P.nll = 0;
  if (plan.mod_mask & (1 << 4)) { P.lla[P.nll] = 2; P.llb[P.nll] = 2; P.nll++; }
  if (plan.mod_mask & ((1 << 6) | (1 << 8))) { P.lla[P.nll] = 4; P.llb[P.nll] = 2; P.nll++; }
  if (plan.mod_mask & (1 << 8)) { P.lla[P.nll] = 4; P.llb[P.nll] = 4; P.nll++; }
  P.nsum = P.nell + P.nll + 2;
  P.need2 = (req_internal & 4) ? 1 : 0;
  P.need4 = (req_internal & 16) ? 1 : 0;
  P.global_los = plan.global_los;
  for (int a = 0; a < 3; ++a) P.los[a] = (float)plan.los[a];
  P.assign = plan.assign;
  P.kf = 2.0 * M_PI / m.box;

  constexpr int NP = row_pad_len<N>();
  const size_t smem = sizeof(C) * (2 * N) + sizeof(T) * (N / 2 + 2) + sizeof(C) * (size_t)(P.nf + 1) * NP;
  auto kern = k_fft_x_contract<T, N>;
  NPC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  NPC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CONTRACT_THREADS, smem));
  if (per_sm < 1) return set_err(ctx, NPC_ERR_UNSUPPORTED, "contraction does not fit on an SM (%zu B smem)", smem);
  const int nrows = (N / 2) * N;
  const int grid = std::min(nrows, per_sm * ctx->num_sms);
  const int nw = CONTRACT_THREADS / 32;
  const size_t nparts = (size_t)grid * nw;
  double* part;
  NPC_TRY(ws_get(ctx, "power.part", sizeof(double) * nparts * P.nbins * P.nsum, (void**)&part));
  NPC_CUDA(ctx, cudaMemsetAsync(part, 0, sizeof(double) * nparts * P.nbins * P.nsum, ctx->stream));
  kern<<<grid, CONTRACT_THREADS, smem, ctx->stream>>>((const C*)half, P, ylm_norm_table(), bintab, (const C*)twp,
                                                      part);
  NPC_LAUNCH(ctx);

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
  for (int l = 0; l <= 4; l += 2) nreq += (plan.ells_mask >> l) & 1;
  F.out_rows = 2 + nreq + F.nmod;
  F.req_mask = plan.ells_mask;
  const int fb = (P.nbins + 127) / 128;
  k_power_finalize<<<fb, 128, 0, ctx->stream>>>(part, F, sc, dev_out);
  NPC_LAUNCH(ctx);
  return NPC_OK;
}

// float32 transforms for 16 <= n <= 1024; float64 transforms for n <= 256
template <typename T>
npc_status fwd_dispatch(npc_ctx* ctx, const PowerPlan& plan, const Geom& g, const void* a, const void* b, void* half) {
  switch (plan.n) {
    case 16: return fwd_impl<T, 16>(ctx, plan, g, a, b, half);
    case 32: return fwd_impl<T, 32>(ctx, plan, g, a, b, half);
    case 64: return fwd_impl<T, 64>(ctx, plan, g, a, b, half);
    case 128: return fwd_impl<T, 128>(ctx, plan, g, a, b, half);
    case 256: return fwd_impl<T, 256>(ctx, plan, g, a, b, half);
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
  }
  if constexpr (sizeof(T) == 4) {
    if (plan.n == 512) return contract_impl<T, 512>(ctx, plan, m, kb, half, sc, out);
    if (plan.n == 1024) return contract_impl<T, 1024>(ctx, plan, m, kb, half, sc, out);
  }
  return set_err(ctx, NPC_ERR_UNSUPPORTED, "mesh size %d not supported at this precision", plan.n);
}

}  // namespace

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
