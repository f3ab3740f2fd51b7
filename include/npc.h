/*
 * npc.h -- C ABI of the GB300 FFT multipole estimator library (libnpc.so).
 *
 * Implements, on one CUDA device, the Fourier-space clustering estimators of Xie et al.,
 * "Efficient estimators for power spectrum and bispectrum multipole measurements":
 *   - Yamamoto power-spectrum multipoles P_l(k) evaluated from the m >= 0 spherical-harmonic
 *     weighted transforms only (Sec. 2.1, Eqs. key1, F_lm_SIC, new_F_ell, pk_final);
 *   - the modified high-order even multipoles P_4b, P_6b, P_8b built from l <= 4 fields
 *     (Sec. 3, Eqs. legendre, Plnew, Pllp);
 *   - Scoccimarro bispectrum multipoles B_l (Sec. 2.2, Eq. bi_sco) and the compressed TripoSH
 *     multipoles B_l0l (Sec. 4, Eq. new_bispec) with their analytic shot noise (Sec. 5.4).
 *
 * Conventions shared by every entry point
 *   Mesh      cubic, n^3 cells, side `box`, covering [origin, origin + box); a particle at
 *             position x has grid coordinate s = (x - origin) * (n / box), evaluated in float64.
 *             Cells are wrapped periodically.  CIC (assign = 2) or TSC (assign = 3); with
 *             interlace = 1 a second mesh assigns s + 1/2 (its point j sits at origin+(j-1/2)H).
 *   Fourier   e^{-i k.x}; W(k) = prod_i sinc(pi k_i / 2k_N)^assign is divided out (Sec. 3.1,
 *             Eq. compensation); the two interlaced meshes are combined as
 *             1/2 [S_a + e^{i H (kx+ky+kz)/2} S_b].
 *   k-bins    modes whose three integer indices lie in (-n/2, n/2), DC excluded, bin
 *             b = floor((k_f |i| - kmin)/dk) with k_f = 2 pi/box (float64), kept if 0 <= b < nbins.
 *   Threads   a context may be used by one host thread at a time.  All device work of a call is
 *             enqueued on the context's stream; calls whose outputs are host memory synchronise
 *             that stream before returning.
 *   Errors    every call returns npc_status; nothing aborts or throws across the ABI.  On error
 *             the outputs are unspecified and npc_last_error() holds a message.  Invalid
 *             arguments are rejected before any device work is enqueued.
 *   Memory    the caller owns every input and output buffer; the context owns and reuses its
 *             device workspace (grown on demand, released by npc_destroy).
 */
#ifndef NPC_H
#define NPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NPC_OK = 0,
  NPC_ERR_INVALID_ARG = 1, /* malformed spec, null pointer, unsupported size or combination */
  NPC_ERR_OOM = 2,         /* device workspace allocation failed */
  NPC_ERR_CUDA = 3,        /* a CUDA runtime call failed (message in npc_last_error) */
  NPC_ERR_UNSUPPORTED = 4, /* valid request outside what this build implements */
  NPC_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  NPC_ERR_NUMERIC = 6      /* non-finite or degenerate normalisation (e.g. empty catalogue) */
} npc_status;

typedef enum { NPC_PREC_FP64 = 0, NPC_PREC_MIXED = 1 } npc_precision;
/* NPC_PREC_FP64: float64 meshes, transforms and sums.  NPC_PREC_MIXED: float32 meshes and
 * transforms, float64 catalogue scalars and k-bin accumulators. */

typedef struct npc_ctx npc_ctx;

/* Mesh, box and line-of-sight specification. */
typedef struct {
  int32_t n;           /* cells per side: a power of two in [16, 1024], or 48, 96, 192 (3 * 2^k) */
  double box;          /* side length of the cubic mesh (length units of the positions) */
  double origin[3];    /* lower corner of the mesh */
  int32_t assign;      /* 2 = CIC, 3 = TSC */
  int32_t interlace;   /* 0 or 1 */
  int32_t periodic;    /* 1: periodic box, no randoms (delta = n - mean); 0: survey with randoms */
  int32_t los;         /* 0: endpoint line of sight xhat from `observer`; 1: global `los_dir` */
  double los_dir[3];   /* used when los == 1 (need not be normalised) */
  double observer[3];  /* used when los == 0 */
} npc_mesh_spec;

/* A catalogue: positions [n][3] (x,y,z interleaved), weights [n], number densities [n]. */
typedef struct {
  const void* pos;     /* required when n > 0 */
  const void* w;       /* NULL: all weights 1 */
  const void* nbar;    /* NULL allowed only where nbar is not used (data catalogue, periodic) */
  int64_t n;           /* number of objects, 0 <= n < 2^31; a catalogue painted with its randoms
                          needs data n + randoms n < 2^31 (NPC_ERR_UNSUPPORTED otherwise) */
  int32_t dtype;       /* 0 = float32, 1 = float64 (all three arrays) */
  int32_t on_device;   /* 1: device pointers on the context's device; 0: host pointers */
} npc_catalog;

/* Half-open bins [kmin + b dk, kmin + (b+1) dk), b = 0..nbins-1; dk > 0, kmin >= 0. */
typedef struct {
  double kmin;
  double dk;
  int32_t nbins;       /* 1 <= nbins <= 4096 */
} npc_kbins;

/* Context ------------------------------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t to enqueue on, or
 * NULL for a stream owned by the context.  The stream must outlive the context. */
npc_status npc_create(npc_ctx** out, int device, void* cuda_stream);
/* Release the context and its device workspace (synchronises its stream).  NULL is accepted. */
npc_status npc_destroy(npc_ctx* ctx);
/* Static string for a status code. */
const char* npc_status_string(npc_status s);
/* Copy the last error message of `ctx` (NUL-terminated, truncated to n bytes). */
npc_status npc_last_error(npc_ctx* ctx, char* buf, size_t n);
/* Library version string "major.minor.patch". */
const char* npc_version(void);

/* Diagnostics of the last completed call on `ctx`. */
typedef struct {
  int32_t n_transforms;        /* Y_lm-weighted forward transforms per mesh phase, counted as in
                                  Table 1 of the paper (one per S_l^m with m >= 0) */
  int32_t n_r2c_equivalent;    /* the same work counted in real-to-complex transforms per phase */
  int32_t n_phases;            /* 1 or 2 (interlacing) */
  int32_t n_kernel_launches;   /* kernels enqueued by the call */
  int64_t workspace_bytes;     /* device workspace held by the context after the call */
  double contraction_flops;    /* bispectrum calls: multiply-add work of the dense triple-product
                                  contractions the call launched, 2 x rows x columns x cells summed
                                  over the launches (the useful products) */
  int32_t contraction_launches;/* number of those launches */
  int32_t reserved;
  double contraction_issued_flops; /* the same contractions as the tensor cores issue them: padded
                                  rows and columns and the parts of the split precision (f16 hi and
                                  lo on the tcgen05 path, tf32 hi*hi + hi*lo + lo*hi on mma.sync) */
} npc_stats;
npc_status npc_last_stats(npc_ctx* ctx, npc_stats* out);

/* Device status of the context (no counterpart in the paper: an operational check).  Kernels
 * whose waits on other threads of their block are bounded (the tensor-core triple products of
 * npc_bispectrum) record NPC_ERR_TIMEOUT in a device word of the context when a wait gives up; the
 * block then waits (with a fixed bound) for its copies and products in flight, frees its tensor
 * memory and exits, so the context stays usable.  The same word records NPC_ERR_NUMERIC when a
 * shell field's largest |value| lies outside [2^-57, 2^63) (other than an all-zero field): the
 * tensor-core path scales its f16 operands by powers of two taken from those maxima, and outside
 * that range they would overflow or lose precision (the mma.sync path has no such limit).  Calls that return host output check the word
 * themselves and return its code; after calls with device output, npc_device_status synchronises
 * the context's stream, returns the recorded code (NPC_OK if none) and clears it. */
npc_status npc_device_status(npc_ctx* ctx);
/* Bound of those waits in GPU clock cycles (<= 0: the default, 2^31 cycles, about a second).  A
 * bound far below the work's latency makes the waits give up: tests use it to exercise the
 * NPC_ERR_TIMEOUT path without any fault. */
npc_status npc_set_wait_limit(npc_ctx* ctx, long long cycles);
/* Implementation switches for comparison runs: "tcgen05_triple" (default 1) selects the tcgen05
 * tensor-core path of the bispectrum triple products (f16 hi + lo operands after exact
 * power-of-two scales, float32 accumulation in tensor memory, launches of more than 32 rows);
 * 0 selects the warp-level mma.sync path (tf32 hi + lo). */
npc_status npc_set_option(npc_ctx* ctx, const char* name, int64_t value);
/* Current value of an option: "tcgen05_triple" as above (npc_batch_tune sets it to the faster path
 * for the batch it times), "batch_branches" (0: not tuned). */
npc_status npc_get_option(npc_ctx* ctx, const char* name, int64_t* value);

/* Stage timing.  With profiling on, every call records CUDA events on the context's stream at its
 * stage boundaries (a few events per call, no synchronisation).  npc_stage_times() waits for the
 * stream, then reports the stages of the last call: names[i] (NUL-terminated, 32 bytes each),
 * ms[i] = device time of stage i and launches[i] = kernels in stage i, for i < *n <= cap. */
npc_status npc_set_profiling(npc_ctx* ctx, int32_t on);
npc_status npc_stage_times(npc_ctx* ctx, char* names, double* ms, int32_t* launches, int32_t cap,
                           int32_t* n);

/* Catalogue scalars (Sec. 2.1, Yamamoto estimator; Sec. 2.2 for I33) --------------------------
 * out[0..7] = { alpha, I22, I33, N0, S3, sum_w(data), sum_w(randoms), sum_w2 } with
 *   alpha = sum_g w / sum_r w,  I22 = alpha sum_r nbar w^2,  I33 = alpha sum_r nbar^2 w^3,
 *   N0 = (sum_g w^2 + alpha^2 sum_r w^2)/I22,  S3 = sum_g w^3 - alpha^3 sum_r w^3,
 *   sum_w2 = sum_g w^2 + alpha^2 sum_r w^2.
 * randoms == NULL means a periodic box of side `box`: alpha = 0, I22 = W^2/V, I33 = W^3/V^2,
 * N0 = sum_g w^2/I22, S3 = sum_g w^3 with W = sum_g w, V = box^3.
 * `out` is host memory when out_on_device == 0, else device memory (then the call is async).
 * Reductions are float64 and bitwise reproducible run to run (fixed reduction order). */
npc_status npc_catalog_scalars(npc_ctx* ctx, const npc_catalog* data, const npc_catalog* randoms,
                               double box, double* out, int32_t out_on_device);

/* Allocation-free catalogue scalars ------------------------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that cannot allocate device
 * memory (a host framework that owns all device memory through its own pool, a plugin that is
 * only handed device pointers, a latency-bound loop that must not pay an allocation's implicit
 * synchronisation).  It computes out[0..7] as npc_catalog_scalars defines them, but needs no
 * context and allocates nothing: its scratch (per-block partial sums) is a static device array of
 * 786,560 bytes that every device which loads the library holds until the process exits.  Its
 * reduction tree depends on n (one block per 4,096 objects, where the context call always sums
 * 1,024 fixed blocks), so the two calls agree to rounding (about 1e-12 relative), not bit for
 * bit; repeated calls on the same inputs are bitwise identical.
 *   - data / randoms: device pointers only (on_device = 1), at most 33,554,432 objects each,
 *     otherwise NPC_ERR_INVALID_ARG with a message in `err`; randoms == NULL means a periodic box.
 *   - out_device: 8 doubles of device memory; the call is asynchronous on `cuda_stream` (NULL:
 *     the legacy default stream) and runs on the calling thread's current device.
 *   - err / errlen: optional buffer for a NUL-terminated message.
 * The first call on each device looks up the address of the static array on that device (again
 * after that device's context changes, e.g. after cudaDeviceReset); make that first call before
 * any stream capture.  Every call reuses the same array and leaves the last call's partial sums
 * in it; calls whose work can overlap on one device (concurrent streams or threads) race on it and
 * must be serialised by the caller.  A launch failure is returned as NPC_ERR_CUDA, and so is an
 * error that earlier asynchronous work left pending (it is not cleared: cudaGetLastError still
 * returns it afterwards). */
npc_status npc_catalog_scalars_noalloc(const npc_catalog* data, const npc_catalog* randoms, double box,
                                       double* out_device, void* cuda_stream, char* err, size_t errlen);

/* Power-spectrum multipoles (Sec. 2.1 Eq. pk_final; Sec. 3 Eqs. Plnew, Pllp) ------------------
 * ell_mask: bit l requests P_l, l in {0, 1, 2, 3, 4}; odd l take the imaginary part of
 * <F_0 F_l^*> (Sec. 2.1), which vanishes for an auto spectrum with a global line of sight.
 * modified_mask: bits 4, 6, 8 request P_4b, P_6b, P_8b (these need the l = 2 and l = 4 fields and
 * are computed from them; Eq. Plnew); bits 16, 17, 18 request the two-index multipoles P_22, P_42,
 * P_44 themselves (Eq. Pllp, shot noise N_ll' subtracted).
 * Output `out` (float64), length npc_power_out_len(), rows of nbins:
 *   [0]            k_eff  = mean |k| over the modes of the bin
 *   [1]            N_modes (number of full-grid modes in the bin)
 *   [2 .. 2+nl)    P_l for the requested l in increasing order, shot noise subtracted (l = 0)
 *   [.. + nm)      P_4b, P_6b, P_8b for the requested ones in increasing order
 *   [.. + nll)     P_22, P_42, P_44 for the requested ones in that order
 *   then 8 scalars as in npc_catalog_scalars.
 * Empty bins report k_eff = N_modes = P = 0.  data->n may be 0 only for a survey (randoms give
 * a zero field and P_0 = -N0); a periodic box needs data->n > 0 (else NPC_ERR_NUMERIC).
 * The transforms are evaluated for m >= 0 only: per mesh phase (l+1) S_l^m fields per l, i.e.
 * 1 + 3 + 5 = 9 for l <= 4 (Table 1); with a global line of sight F_l(k) = L_l(khat.los) F_0(k)
 * and a single transform suffices. */
npc_status npc_power_multipoles(npc_ctx* ctx, const npc_mesh_spec* mesh, const npc_catalog* data,
                                const npc_catalog* randoms, const npc_kbins* bins,
                                uint32_t ell_mask, uint32_t modified_mask, npc_precision prec,
                                double* out, int32_t out_on_device);
/* Number of doubles written by npc_power_multipoles for this request (0 if the masks are bad). */
int64_t npc_power_out_len(const npc_kbins* bins, uint32_t ell_mask, uint32_t modified_mask);

/* Cross multipoles of two tracers A and B (multi-tracer spectra, which the paper's toolkit
 * measures alongside the auto spectra; Sec. 6) -----------------------------------------------
 * P_l^AB(k) = (2l+1)/I22^AB <Re F_0^A(k) F_l^B*(k)>_bin with F_l^B the m >= 0 Yamamoto field of
 * tracer B (its line of sight: observer to B's grid points, or the global los), F_0^A the FKP field
 * of A, I22^AB = sqrt(I22^A I22^B), and no shot noise subtracted (the tracers share no object).
 * Both tracers use the same mesh spec; randoms_a and randoms_b are both NULL (periodic box) or both
 * given (survey).  ell_mask: bits 0 .. 4.  Cost: B's transforms plus one per phase for A.
 * Output as npc_power_multipoles with modified_mask = 0 (length npc_power_out_len(bins, ell_mask,
 * 0)), the 8 trailing scalars being [alpha_A, I22^AB, alpha_B, 0, I22^A, I22^B, sum w_A, sum w_B].
 * ell_mask may include the odd bits 1, 3 (imaginary part, as for npc_power_multipoles).
 * Errors: as npc_power_multipoles; NPC_ERR_NUMERIC for an empty catalogue of either tracer. */
npc_status npc_cross_power_multipoles(npc_ctx* ctx, const npc_mesh_spec* mesh, const npc_catalog* data_a,
                                      const npc_catalog* randoms_a, const npc_catalog* data_b,
                                      const npc_catalog* randoms_b, const npc_kbins* bins, uint32_t ell_mask,
                                      npc_precision prec, double* out, int32_t out_on_device);

/* Bispectrum multipoles (Sec. 2.2 Eq. bi_sco; Sec. 4 Eq. new_bispec; Sec. 5.4 shot noise) ------
 * Periodic box (mesh->periodic = 1, randoms = NULL) with a global line of sight (mesh->los = 1) for l = 2;
 * survey geometry (mesh->periodic = 0, randoms required): the monopoles need no line of sight; for
 * l = 2 either the global one (los = 1) or the line of sight from mesh->observer to each grid point
 * (los = 0), where X_2 is the Yamamoto field of Eq. hand from Y_2m-weighted transforms (the
 * compressed B_202 carries it on the k3 leg) and the analytic shot noise uses the Yamamoto N-field
 * and the catalogue moments sum_p w_p^3 Y_2m(xhat_p) for its self term (shot = 2 is not available
 * there: NPC_ERR_UNSUPPORTED).
 * Triangles: bins i <= j <= k closing at their centres, c_k <= c_i + c_j, c_b = kmin+(b+1/2)dk,
 * in lexicographic (i, j, k) order; pairs: i <= j in lexicographic order.  The largest bin edge
 * must not exceed k_N/2 (the closure would alias otherwise), else NPC_ERR_UNSUPPORTED.
 * scoc_ell_mask: bits 0, 1, 2, 3 request B_0, B_1, B_2, B_3 (l on the first, smallest side).  The odd
 *   multipoles follow Sec. 2.1's rule for odd l: X_l is anti-Hermitian, its shell fields are i A_b(x),
 *   and B_l reports the imaginary part (2l+1)/(I33 N_T) sum_x A_i F_j F_k / N^3; with the line of
 *   sight to each grid point X_l is the Yamamoto field of the Y_lm-weighted transforms, with a global
 *   line of sight L_l(qhat . los) X_0.  They are raw estimates: their shot noise is reported as 0.
 * tripo_ell_mask: bits 0, 2 request the compressed B_000, B_202.
 * shot: 1 subtracts the analytic shot noise (Sec. 5.4, thin-shell integrals) and reports it;
 *   2 uses the FFT method instead (Sec. 5.4.2): the exact sums of the two-object terms over the
 *   closed triplets of B_l (sum_x I_a I_b G_c with shell fields G_c of X_0 N_0^*, L_2-weighted
 *   indicators for l = 2) and over the bin pairs of B_l0l (full-range fields of L_l X_0 N_0^* and of
 *   L_l), about twice the triple-product work; 0 leaves the raw estimates.
 * Output `out` (float64), length from npc_bispectrum_layout():
 *   [ns][ntri]  B_l          [ns][ntri]  shot noise of B_l      [ntri] N_T (closed triplets)
 *   [nt][npair] B_l0l        [nt][npair] shot noise of B_l0l    [nbins] N_modes
 *   then 8 scalars as in npc_catalog_scalars. */
npc_status npc_bispectrum(npc_ctx* ctx, const npc_mesh_spec* mesh, const npc_catalog* data,
                          const npc_catalog* randoms, const npc_kbins* bins,
                          uint32_t scoc_ell_mask, uint32_t tripo_ell_mask, int32_t shot,
                          npc_precision prec, double* out, int32_t out_on_device);
/* Multi-tracer bispectra (Sec. 6 lists auto and cross bispectra; the cross form is this library's
 * reading): three tracers, tracer 1 on leg 1 (k1, which carries the line of sight of B_l), tracers
 * 2 and 3 on legs 2 and 3 (on k3 for B_l0l):
 *   B_l^{123}(i,j,k) = (2l+1)/(I33^{123} N_T) sum_closed L_l(mu1) X^1(q1) X^2(q2) X^3(q3)
 *   B_l0l^{123}(i,j) = (2l+1)/(I33^{123} N_i N_j) sum_{q1 in i, q2 in j} X^1(q1) X^2(q2) L_l(mu3) X^3(q3)
 * with I33^{123} = (I33^1 I33^2 I33^3)^(1/3) (exact when the three selections n w share a shape).
 * data: array of 3 catalogues; randoms: NULL (periodic box) or an array of 3.  A global line of
 * sight is required (mesh->los = 1).  scoc_ell_mask, tripo_ell_mask: bits 0 and 2.  Raw estimates:
 * no shot noise is subtracted (a pair of legs on one tracer would carry one) and the shot-noise
 * entries of the output are 0.  Output layout, triangle and pair order as npc_bispectrum (the 8
 * scalars are tracer 1's, with I33 replaced by I33^{123} and S3 by 0). */
npc_status npc_cross_bispectrum(npc_ctx* ctx, const npc_mesh_spec* mesh, const npc_catalog* data,
                                const npc_catalog* randoms, const npc_kbins* bins, uint32_t scoc_ell_mask,
                                uint32_t tripo_ell_mask, npc_precision prec, double* out, int32_t out_on_device);
/* Sizes for npc_bispectrum.  Any output pointer may be NULL. */
npc_status npc_bispectrum_layout(const npc_kbins* bins, uint32_t scoc_ell_mask,
                                 uint32_t tripo_ell_mask, int64_t* ntri, int64_t* npairs,
                                 int64_t* out_len);
/* Triangle bin indices [ntri][3] in npc_bispectrum's order (host memory, capacity `cap` triangles).
 * *ntri receives the count; tri = NULL only asks for it; cap below the count returns
 * NPC_ERR_INVALID_ARG and writes nothing to tri. */
npc_status npc_bispectrum_triangles(const npc_kbins* bins, int32_t* tri, int64_t cap,
                                    int64_t* ntri);

/* Sugiyama TripoSH bispectrum multipoles B_{l1 l2 L}(k1, k2) (Sec. 4.2, Eq. sugi_estimator with the
 * fields of Eq. F_and_G).  Global line of sight (mesh->periodic = 1, or survey geometry with randoms
 * and mesh->los = 1):
 *   B(i, j) = H N / (I33 N_i N_j) sum_{m1 m2 M} (l1 l2 L; m1 m2 M) <F_l1^m1(x; k_i) F_l2^m2(x; k_j) G_L^M(x)>_x
 * with F_l^m(x; k) = sum_{q in bin k} e^{iqx} y_l^{m*}(qhat) X(q), H = (l1 l2 L; 0 0 0),
 * N = (2l1+1)(2l2+1)(2L+1), y = sqrt(4 pi/(2l+1)) Y, X the compensated interlaced spectrum and
 * <.>_x the mean over the grid.  In the frame whose third axis is the line of sight only M = 0
 * remains, G_L^0 is the full-range field of X for every L, and the m, -m sub-configurations pair up
 * (Eq. sym_sugi): the library evaluates sum_{m=0..min(l1,l2)} of the real parts of F_l1^m F_l2^{m*} G
 * as shell-field triple products on the tensor cores, every (k_i, k_j) bin pair at once.
 * Survey geometry with the line of sight to each grid point (mesh->los = 0, randoms required): the
 *   full sum over (m1, m2, M = -m1-m2) in the catalogue frame, G_L^M(x) = sum_q e^{iqx} dn_L^M(q)/W(q)
 *   with dn_L^M the interlaced transform of F(x) y_L^{M*}(xhat) (xhat from mesh->observer to the grid
 *   point), from the transforms of F Re Y_LM and F Im Y_LM for M >= 0 (G_L^{-M} = (-1)^M G_L^{M*});
 *   every sub-configuration becomes real triple products of the parts of F_l1^|m1|, F_l2^|m2| and
 *   G_L^|M|.  For l1 + l2 odd (odd L) the sum is imaginary and its imaginary part is reported (the
 *   rule of Sec. 2.1 for odd multipoles).  Raw estimates only there (shot = 0, else
 *   NPC_ERR_UNSUPPORTED).
 * multipoles: nmult (1..16) triples (l1, l2, L), 0 <= l1, l2 <= 4, |l1 - l2| <= L <= l1 + l2; with a
 *   global line of sight L and l1 + l2 even (the plane-parallel symmetry about it), with the line of
 *   sight to each grid point l1 + l2 + L even and L <= 4; else NPC_ERR_INVALID_ARG.  Bins and mesh
 *   limits as npc_bispectrum (at most 24 bins, largest bin edge <= k_N/2).
 * shot: 0 raw estimates; 1 subtracts the analytic shot noise of Sec. 5.4 and reports it:
 *   delta_{l1 0} delta_{l2 0} delta_{L 0} S/I33 (three legs from one object), delta_{l1 L} delta_{l2 0}
 *   (2L+1) H_L(k1)/I33 and delta_{l2 L} delta_{l1 0} (2L+1) H_L(k2)/I33 (two), and for legs 1, 2 from
 *   one object the thin-shell ring average of Lemma 1, H N/I33 sum_k3 w q_{l1 l2 L}(k1, k2, k3)
 *   Q_L(k3) / sum_k3 w over the shells of width dk that close the pair (w = N_mode/k3), with
 *   H_L = Q_L = <L_L(mu) Re X N^*> - S <L_L(mu)> on the k-bins and the k3 shells (N the w^2 field)
 *   and q built from Racah-normalised associated Legendre functions; 2 uses the FFT method of
 *   Sec. 5.4.2 instead (exact): legs 1, 2 from one object as triple products of the y_l^m-weighted
 *   indicator shells against the full-range field of X N^*, legs 1, 3 and 2, 3 and the pure term as
 *   products of per-bin sums A_l^m = sum y_l^{m*}(qhat) and C_l^m = sum y_l^{m*}(qhat) X N^*,
 *   shot = H N/(I33 N_i N_j) sum_m (l1 l2 L; m -m 0) Re[T12 + A1 C2 + C1 A2 - 2 S A1 A2].
 * Output `out` (float64, host or device as out_on_device), length npc_bispectrum_sugiyama_len():
 *   [nmult][nbins][nbins] B (k1 = bin i the row, k2 = bin j the column; raw minus shot noise),
 *   [nmult][nbins][nbins] shot noise (zeros when shot = 0), [nbins] N_modes, then 8 scalars as in
 *   npc_catalog_scalars.
 * Errors as npc_bispectrum; shot other than 0, 1 or 2: NPC_ERR_INVALID_ARG. */
npc_status npc_bispectrum_sugiyama(npc_ctx* ctx, const npc_mesh_spec* mesh, const npc_catalog* data,
                                   const npc_catalog* randoms, const npc_kbins* bins, int32_t nmult,
                                   const int32_t* multipoles, int32_t shot, npc_precision prec,
                                   double* out, int32_t out_on_device);
/* Output length of npc_bispectrum_sugiyama: 2 nmult nbins^2 + nbins + 8 (-1 for bad arguments). */
int64_t npc_bispectrum_sugiyama_len(const npc_kbins* bins, int32_t nmult);

/* Batches of measurements --------------------------------------------------------------------------
 * Many mocks of uneven catalogue size and mesh, each measured as npc_power_multipoles (P_l for
 * ell_mask, no modified multipoles) and, when bispec_bins.nbins > 0, as npc_bispectrum with the
 * Scoccimarro monopole B_0 and its analytic shot noise (scoc_ell_mask = 1, tripo_ell_mask = 0,
 * shot = 1; periodic boxes and survey geometry).  The paper measures its estimators mock by mock;
 * the batch changes only how the work is scheduled, not what is computed: every item's output
 * equals, bit for bit, the single call on the same inputs.
 * Items run on concurrent branches (private streams and workspaces of the context); with
 * NPC_BATCH_GRAPH the first call of a batch shape also captures the whole sequence into a CUDA
 * graph, and later calls with identical items (same pointers, sizes and specs) and the same
 * output pointer replay it with one graph launch.  Catalogues must be device memory that stays
 * valid (and may be refilled in place) while graphs of them are replayed. */
#define NPC_BATCH_GRAPH 1

typedef struct {
  npc_mesh_spec mesh;
  npc_catalog data;          /* device memory, n > 0 */
  npc_catalog randoms;       /* device memory for a survey; n = 0 for a periodic box */
  npc_kbins power_bins;
  npc_kbins bispec_bins;     /* nbins = 0: no bispectrum; else largest edge <= k_N/2, nbins <= 24 */
} npc_batch_item;

/* Total output length in doubles for the batch (0 for a bad request); offsets[2i] and offsets[2i+1]
 * (may be NULL) receive the start of item i's P_l block (layout of npc_power_multipoles) and of its
 * B_0 block (layout of npc_bispectrum with one Scoccimarro multipole and no compressed one), or -1. */
int64_t npc_batch_layout(int32_t nitems, const npc_batch_item* items, uint32_t ell_mask,
                         int64_t* offsets);
/* Run the batch; out_device (device memory, npc_batch_layout() doubles) receives every item's
 * block.  Asynchronous on the context's stream.  flags: 0 or NPC_BATCH_GRAPH. */
npc_status npc_batch_run(npc_ctx* ctx, int32_t nitems, const npc_batch_item* items, uint32_t ell_mask,
                         npc_precision prec, double* out_device, int32_t flags);
/* Autotuner: times, on this batch, the columns per CTA of the y transform pass for every mesh size,
 * then the number of concurrent branches (graph replays), then the triple-product path of the
 * bispectra (tcgen05 tiles of 128 rows or warp-level tiles of 16 rows, option "tcgen05_triple"),
 * keeps the fastest choices in the context and reports the branch count.  Runs the batch several
 * times (out_device is overwritten).  After a batch, npc_device_status also checks the bounded
 * waits of the batch's branch contexts. */
npc_status npc_batch_tune(npc_ctx* ctx, int32_t nitems, const npc_batch_item* items, uint32_t ell_mask,
                          npc_precision prec, double* out_device, int32_t* branches);
/* Autotuner of the transform passes for mesh size n: times the valid column-tile widths of the
 * y pass on a scratch buffer and keeps the fastest for (n, prec) in the context; every later call
 * on the context uses it.  Synchronous; results do not depend on the choice (same arithmetic per
 * column). */
npc_status npc_tune_transforms(npc_ctx* ctx, int32_t n, npc_precision prec);
/* Fix the number of concurrent branches (1..16; 0 restores the default of 4). */
npc_status npc_batch_set_branches(npc_ctx* ctx, int32_t branches);

/* Mesh-level estimators and their adjoints ------------------------------------------------------
 * The paper defines its estimators as functions of the density field (Sec. 2.1 Eq. pk_final for
 * P_l; Sec. 2.2 Eq. bi_sco for B_l) but does not differentiate them.  These calls expose the same
 * estimators on a caller-owned mesh, and their exact derivatives, so the measurement can sit inside
 * a gradient-based fit.  Scope: periodic box, global line of sight, one mesh without interlacing
 * (spec->periodic = 1, spec->los = 1, spec->interlace = 0), else NPC_ERR_UNSUPPORTED.
 *
 * Mesh layout: n^3 values of the precision's type (float32 for NPC_PREC_MIXED, float64 for
 * NPC_PREC_FP64), index (z n + y) n + x, device memory of the context's device.
 * With X(q) = sum_x delta(x) e^{-iq.x} / W(q) and the bins of npc_power_multipoles:
 *   P_l(b) = (2l+1)/(I22 N_b) sum_{q in b} L_l(qhat.los) |X(q)|^2 - delta_l0 N0,   l in {0, 2, 4};
 *   B_0(b) = sum_x F_b(x)^3 / (I33 sum_x I_b(x)^3),  F_b(x) = sum_{q in b} X(q) e^{iq.x},
 *            I_b(x) = sum_{q in b} e^{iq.x}   (the equilateral triangle (b, b, b) of Eq. bi_sco).
 * I22, N0 and I33 are inputs (npc_catalog_scalars gives them for a catalogue); they are held fixed
 * under differentiation.  B_0 needs the largest bin edge <= k_N/2 and nbins <= 32. */

/* Number of doubles npc_mesh_multipoles writes (0 for a bad request). */
int64_t npc_mesh_multipoles_len(const npc_kbins* bins, uint32_t ell_mask, int32_t b0);

/* Forward values.  ell_mask: bits 0, 2, 4 request P_l; b0 = 1 requests B_0.  Output rows of
 * nbins: [0] k_eff, [1] N_modes, then P_l for the requested l in increasing order, then (b0) B_0
 * and N_T (closed wavevector triples of the equilateral bin triangle).  `out` is host memory when
 * out_on_device == 0 (the call then synchronises), else device memory.  Sums are float64 and
 * reproducible run to run. */
npc_status npc_mesh_multipoles(npc_ctx* ctx, const npc_mesh_spec* spec, const void* mesh,
                               const npc_kbins* bins, uint32_t ell_mask, int32_t b0, double i22,
                               double n0, double i33, npc_precision prec, double* out,
                               int32_t out_on_device);

/* Vector-Jacobian product: grad_mesh(x) = dL/ddelta(x) for the loss with cotangents
 * dl_dp[e][b] = dL/dP_{l_e}(b) (requested l in increasing order) and dl_db0[b] = dL/dB_0(b):
 *   dL/ddelta(x) = sum_q [2 K(q) X(q) + sum_b c_b Phi_b(q) D_b(q)] / W(q) e^{iq.x},
 *   K(q) = sum_{l,b} dl_dp (2l+1) Phi_b(q) L_l(qhat.los) / (I22 N_b),
 *   c_b = 3 dl_db0[b] / (I33 sum_x I_b^3),  D_b(q) = sum_x F_b(x)^2 e^{-iq.x}.
 * The transforms are recomputed from `mesh` (nothing is kept from the forward call).
 * Cotangents are host (cotangents_on_device = 0) or device memory; grad_mesh is device memory in
 * the mesh layout and is overwritten. */
npc_status npc_mesh_multipoles_vjp(npc_ctx* ctx, const npc_mesh_spec* spec, const void* mesh,
                                   const npc_kbins* bins, uint32_t ell_mask, int32_t b0,
                                   double i22, double i33, const double* dl_dp,
                                   const double* dl_db0, int32_t cotangents_on_device,
                                   npc_precision prec, void* grad_mesh);

/* Deterministic mass assignment of a periodic catalogue onto one mesh (spec->periodic = 1,
 * spec->interlace = 0): mesh(c) = sum_p w_p W(c - s_p) - sum_p w_p / n^3, in the mesh layout above
 * (device memory, overwritten).  The same painting as the estimator calls. */
npc_status npc_paint_mesh(npc_ctx* ctx, const npc_mesh_spec* spec, const npc_catalog* data,
                          npc_precision prec, void* mesh);

/* Adjoint of npc_paint_mesh with respect to positions and weights, for a cotangent mesh G:
 *   grad_pos[p][a] = w_p (n/box) sum_c G(c) dW(c - s_p)/ds_a,   grad_w[p] = sum_c G(c) W(c - s_p),
 * over the 8 (CIC) or 27 (TSC) taps, with the tap cells decided in float64 as in the forward
 * assignment (the window is piecewise polynomial; at a cell boundary the one-sided derivative of the
 * chosen taps is returned).  The catalogue must be on the device; grad_pos ([n][3]) and grad_w ([n],
 * may be NULL) are device arrays of the catalogue's dtype; grad_mesh has the precision's type. */
npc_status npc_paint_adjoint(npc_ctx* ctx, const npc_mesh_spec* spec, const npc_catalog* data,
                             const void* grad_mesh, npc_precision prec, void* grad_pos,
                             void* grad_w);

/* Single-purpose forms (float32 meshes, NPC_PREC_MIXED, device memory, host cotangents):
 *   npc_power_vjp   = npc_mesh_multipoles_vjp with b0 = 0 (dl_dp[e][b] for the requested l);
 *   npc_bispec0_vjp = npc_mesh_multipoles_vjp with ell_mask = 0, b0 = 1;
 *   npc_tsc_adjoint = npc_paint_adjoint for TSC (spec->assign = 3, else NPC_ERR_INVALID_ARG),
 *                     positions only (grad_pos of the catalogue's dtype). */
npc_status npc_power_vjp(npc_ctx* ctx, const float* delta, const npc_mesh_spec* spec, const npc_kbins* bins,
                         uint32_t ell_mask, double i22, const double* dl_dp, float* dl_ddelta);
npc_status npc_bispec0_vjp(npc_ctx* ctx, const float* delta, const npc_mesh_spec* spec, const npc_kbins* bins,
                           double i33, const double* dl_db0, float* dl_ddelta);
npc_status npc_tsc_adjoint(npc_ctx* ctx, const npc_mesh_spec* spec, const npc_catalog* data, const float* grad_mesh,
                           void* grad_pos);

#ifdef __cplusplus
}
#endif
#endif /* NPC_H */
