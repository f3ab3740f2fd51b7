// Internal declarations shared by the translation units of libnpc.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "../../include/npc.h"

// ---------------------------------------------------------------------------------------------
// Complex helpers (float2 / double2)
// ---------------------------------------------------------------------------------------------
template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename T> using cplx = typename CplxOf<T>::type;

__host__ __device__ __forceinline__ float2 cmk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 cmk(double a, double b) { return make_double2(a, b); }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return cmk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return cmk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return cmk(a.x, -a.y); }
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) {
  return cmk(a.x * s, a.y * s);
}
// multiply by (sign * i): sign = -1 gives -i, +1 gives +i
template <int SIGN, typename C> __host__ __device__ __forceinline__ C cmul_i(C a) {
  return SIGN < 0 ? cmk(a.y, -a.x) : cmk(-a.y, a.x);
}

// ---------------------------------------------------------------------------------------------
// Spherical harmonics Y_l^m (m >= 0, Condon-Shortley phase) at a unit vector, l <= 8.
//   Y_l^m = N_lm Q_lm(z) (x + i y)^m,  N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
//   Q_lm = (-1)^m d^m L_l/dz^m, from Q_mm = (-1)^m (2m-1)!!, Q_{m+1,m} = (2m+1) z Q_mm and the
//   three-term recurrence (l-m) Q_lm = (2l-1) z Q_{l-1,m} - (l+m-1) Q_{l-2,m}.
// ---------------------------------------------------------------------------------------------
constexpr int NPC_LMAX = 8;
constexpr int NPC_NLM = (NPC_LMAX + 1) * (NPC_LMAX + 2) / 2;

struct YNorm {
  double v[NPC_NLM];  // index l(l+1)/2 + m
  float f[NPC_NLM];   // the same, rounded once to float (no float64 work in float kernels)
};
YNorm ylm_norm_table();
template <typename T> __device__ __forceinline__ T ynorm(const YNorm& n, int i);
template <> __device__ __forceinline__ float ynorm<float>(const YNorm& n, int i) { return n.f[i]; }
template <> __device__ __forceinline__ double ynorm<double>(const YNorm& n, int i) { return n.v[i]; }

template <typename T>
__device__ __forceinline__ void ylm_eval(int l, int m, T x, T y, T z, const YNorm& nrm, T& re, T& im) {
  T pr = T(1), pim = T(0);
  for (int j = 0; j < m; ++j) {
    const T nr = pr * x - pim * y;
    pim = pr * y + pim * x;
    pr = nr;
  }
  T qmm = T(1);
  for (int j = 1; j <= m; ++j) qmm *= -T(2 * j - 1);
  T q = qmm;
  if (l > m) {
    T q0 = qmm;
    T q1 = z * T(2 * m + 1) * qmm;
    for (int ll = m + 2; ll <= l; ++ll) {
      const T q2 = (T(2 * ll - 1) * z * q1 - T(ll + m - 1) * q0) / T(ll - m);
      q0 = q1;
      q1 = q2;
    }
    q = q1;
  }
  const T c = ynorm<T>(nrm, l * (l + 1) / 2 + m) * q;
  re = c * pr;
  im = c * pim;
}

// Closed forms of Q_lm for l in {2, 4} (expanded from the recurrence above), falling back to
// the recurrence otherwise.  (x, y, z) is a unit vector.
template <typename T>
__device__ __forceinline__ void ylm_fast(int l, int m, T x, T y, T z, const YNorm& nrm, T& re, T& im) {
  const T z2 = z * z;
  T q;
  switch (l * 16 + m) {
    case 0x00: re = ynorm<T>(nrm, 0); im = T(0); return;
    case 0x20: q = T(1.5) * z2 - T(0.5); break;
    case 0x21: q = T(-3) * z; break;
    case 0x22: q = T(3); break;
    case 0x40: q = (T(35) * z2 * z2 - T(30) * z2 + T(3)) * T(0.125); break;
    case 0x41: q = T(-2.5) * z * (T(7) * z2 - T(3)); break;
    case 0x42: q = T(7.5) * (T(7) * z2 - T(1)); break;
    case 0x43: q = T(-105) * z; break;
    case 0x44: q = T(105); break;
    default: ylm_eval<T>(l, m, x, y, z, nrm, re, im); return;
  }
  T pr = T(1), pim = T(0);
  for (int j = 0; j < m; ++j) {
    const T nr = pr * x - pim * y;
    pim = pr * y + pim * x;
    pr = nr;
  }
  const T c = ynorm<T>(nrm, l * (l + 1) / 2 + m) * q;
  re = c * pr;
  im = c * pim;
}

// Legendre polynomial L_l(mu), l <= 8 (Bonnet recurrence).
template <typename T> __device__ __forceinline__ T legendre_p(int l, T mu) {
  if (l == 0) return T(1);
  T p0 = T(1), p1 = mu;
  for (int ll = 2; ll <= l; ++ll) {
    const T p2 = (T(2 * ll - 1) * mu * p1 - T(ll - 1) * p0) / T(ll);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// ---------------------------------------------------------------------------------------------
// Field descriptors for the forward transforms
// ---------------------------------------------------------------------------------------------
enum : int8_t { PART_RE = 0, PART_IM = 1, PART_ONE = 2, PART_ZERO = 3 };

struct Comp {          // one real field: mesh phase x weight function
  int8_t phase;        // 0 or 1
  int8_t ell, m;       // Y_l^m (m >= 0)
  int8_t part;         // PART_RE / PART_IM of Y_l^m, PART_ONE (global LOS), PART_ZERO
  int8_t tracer = 0;   // 1: F_0 of the first tracer A of a cross spectrum (the others are B's)
};

constexpr int NPC_MAX_FIELDS = 56;  // real fields per call (2 phases x 25 for l = 0 .. 4, + tracer A)

struct FieldList {
  int nf;                     // number of real fields
  Comp f[NPC_MAX_FIELDS];     // real field f; forward pairs are (2p, 2p+1)
};

// Geometry needed to evaluate xhat at a grid point.
struct Geom {
  int n;
  double h;          // box / n
  double o[3];       // origin - observer
  double los[3];     // unit global LOS
  int global_los;
};

// ---------------------------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------------------------
struct Workspace {
  void* p = nullptr;
  size_t bytes = 0;
};

struct npc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  std::map<std::string, Workspace> ws;
  std::map<std::string, std::vector<char>> host_cache_keys;
  std::string last_error;
  npc_stats stats{};
  int launches = 0;
  double contraction_flops = 0.0;   // dense triple-product work of the current call
  int contraction_launches = 0;
  double contraction_issued_flops = 0.0;   // the same work as the tensor cores issue it (padding, split parts)
  // device status word written by kernels whose waits are bounded (0 = fine, else an npc_status),
  // the wait bound they are given (clock cycles) and whether the current call launched one
  int* dev_status = nullptr;
  long long wait_limit = 0;          // <= 0: the default bound
  bool bounded_waits = false;
  // triple products on the tcgen05 tensor cores (off: the mma.sync path), for comparison runs
  bool use_tcgen05 = true;
  // stage profiling (events recorded on `stream` at stage boundaries when enabled)
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::string> stage_names;
  std::vector<int> stage_launches;
  int ev_used = 0;
  int launches_at_mark = 0;
  // batches: cached device tables are named per measurement slot so that a captured graph of
  // many measurements never re-uploads a table; while capturing, workspace growth and table
  // uploads are errors (the warm-up run sizes everything first)
  int slot_base = 0;
  bool capturing = false;
  uint64_t ws_generation = 0;          // bumped whenever a workspace buffer moves
  std::vector<npc_ctx*> subs;          // per-branch contexts of the batch executor
  std::map<std::string, struct BatchGraph*> graphs;
  int batch_branches = 0;              // 0: not tuned (default 4)
  std::map<int, int> ytx;              // tuned columns per CTA of the y pass, per (n * 2 + fp64)
  cudaStream_t batch_hub = nullptr;    // stream the batch graphs are captured on and launched from
};

// default bound of a device-side wait: about one second at the GPU's clock
constexpr long long NPC_DEFAULT_WAIT_CYCLES = 1ll << 31;
inline long long wait_cycles(const npc_ctx* ctx) {
  return ctx->wait_limit > 0 ? ctx->wait_limit : NPC_DEFAULT_WAIT_CYCLES;
}
// reads (and clears) the device status word after a synchronisation of the context's stream
npc_status check_device_status(npc_ctx* ctx);

// releases branch contexts, graphs and the batch stream (batch.cu)
void destroy_batch_state(npc_ctx* ctx);

// slot-qualified name of a cached table or cache entry
std::string slot_name(const npc_ctx* ctx, const std::string& name);

// Marks the end of a stage named `name` (and the start of the next) when profiling is on.
npc_status stage_mark(npc_ctx* ctx, const char* name);
npc_status stage_begin(npc_ctx* ctx);

// error helpers
npc_status set_err(npc_ctx* ctx, npc_status s, const char* fmt, ...);
#define NPC_CUDA(ctx, call)                                                                  \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return set_err((ctx), NPC_ERR_CUDA, "%s failed: %s (%s:%d)", #call,                    \
                     cudaGetErrorString(e_), __FILE__, __LINE__);                            \
  } while (0)
#define NPC_LAUNCH(ctx)                                                                      \
  do {                                                                                       \
    (ctx)->launches++;                                                                       \
    cudaError_t e_ = cudaGetLastError();                                                     \
    if (e_ != cudaSuccess)                                                                   \
      return set_err((ctx), NPC_ERR_CUDA, "kernel launch failed: %s (%s:%d)",                \
                     cudaGetErrorString(e_), __FILE__, __LINE__);                            \
  } while (0)
#define NPC_TRY(expr)                                                                        \
  do {                                                                                       \
    npc_status s_ = (expr);                                                                  \
    if (s_ != NPC_OK) return s_;                                                             \
  } while (0)

// grow-only named device buffer
npc_status ws_get(npc_ctx* ctx, const char* name, size_t bytes, void** out);
// cached device table keyed by (name, key bytes); uploads `data` on first use
npc_status ws_table(npc_ctx* ctx, const std::string& name, const std::vector<char>& key,
                    const void* data, size_t bytes, void** out);

// Shared host helpers of the public entry points (api.cu)
npc_status check_spec(npc_ctx* ctx, const npc_mesh_spec* m);
npc_status check_catalog(npc_ctx* ctx, const npc_catalog* c, const char* what, bool need_nbar);
npc_status check_painted_pair(npc_ctx* ctx, const npc_catalog* d, const npc_catalog* r);
npc_status check_bins(npc_ctx* ctx, const npc_kbins* b);
struct DevCatalog;
npc_status stage_catalog(npc_ctx* ctx, const npc_catalog* c, const char* tag, DevCatalog* out);
Geom make_geom(const npc_mesh_spec& m);
void begin_call(npc_ctx* ctx);
npc_status end_call(npc_ctx* ctx);
npc_status finish_output(npc_ctx* ctx, const double* dev, double* out, int64_t len, int out_on_device);

// ---------------------------------------------------------------------------------------------
// Scalars layout in device memory (double[16])
// ---------------------------------------------------------------------------------------------
enum {
  SC_ALPHA = 0, SC_I22, SC_I33, SC_N0, SC_S3, SC_SUMWG, SC_SUMWR, SC_SUMW2,
  SC_MAXW_F = 8,   // max |weight coefficient| for the FKP field (data w, randoms alpha w)
  SC_MAXW_N = 9,   // same for the w^2 N-field
  SC_COUNT = 16
};

// ---------------------------------------------------------------------------------------------
// Host launchers (catalog.cu)
// ---------------------------------------------------------------------------------------------
struct DevCatalog {   // catalogue resident on the device
  const void* pos = nullptr;
  const void* w = nullptr;
  const void* nbar = nullptr;
  int64_t n = 0;
  int dtype = 0;      // 0 float, 1 double
};

npc_status launch_catalog_scalars(npc_ctx* ctx, const DevCatalog& d, const DevCatalog* r, double box,
                                  double* dev_scalars);
// Cross-spectrum scalars from tracers A and B (output slots documented with npc_cross_power_multipoles).
npc_status launch_cross_scalars(npc_ctx* ctx, const double* sa, const double* sb, double* sx);
npc_status launch_cross3_scalars(npc_ctx* ctx, const double* s1, const double* s2, const double* s3, double* sx);

// Paint the FKP field (weight_power 1) or the N-field (2) on 1 or 2 interlacing phases.
// meshes: nphase pointers to n^3 arrays of T (layout [z][y][x]).
npc_status launch_paint(npc_ctx* ctx, const DevCatalog& d, const DevCatalog* r, const npc_mesh_spec& m,
                        int weight_power, int prec, const double* dev_scalars, void* mesh_a,
                        void* mesh_b);

// ---------------------------------------------------------------------------------------------
// Power spectrum passes (power.cu)
// ---------------------------------------------------------------------------------------------
struct PowerPlan {
  int n;
  int nphase;
  FieldList fl;
  int ells_mask;        // requested P_l
  int mod_mask;         // requested P_lb
  int need_ll;          // 1: two-index sums needed
  int nbins;
  int nsum;             // sums per bin
  int global_los;
  double los[3];
  int assign;
  int kz_keep;          // forward passes keep kz < kz_keep (0: all, n/2)
  int row_n2max;        // > 0: the y pass may skip rows (ky, kz) with ky^2 + kz^2 above it
  int cross;            // 1: cross spectrum, P_l = Re<F_0^A F_l^B*> with A's fields marked `tracer`
};

// Catalogue -> P_l after validation, staging and the catalogue scalars `sc` (api.cu).
npc_status power_core(npc_ctx* ctx, const npc_mesh_spec& ms, const DevCatalog& d, const DevCatalog* r,
                      const npc_kbins& kb, uint32_t ell_mask, uint32_t modified_mask, int prec, const double* sc,
                      double* dev_out);

// Autotuner of the y pass (columns per CTA) for mesh size n; the choice is kept in ctx->ytx.
npc_status tune_y_pass(npc_ctx* ctx, int n, int prec, int nplanes);

npc_status run_forward_transforms(npc_ctx* ctx, int prec, const PowerPlan& plan, const Geom& g,
                                  const void* mesh_a, const void* mesh_b, void* half);
npc_status run_power_contract(npc_ctx* ctx, int prec, const PowerPlan& plan, const npc_mesh_spec& m,
                              const npc_kbins& kb, const void* half, const double* dev_scalars,
                              double* dev_out);

// bin table: int16 per integer |k|^2 in [0, 3 (n/2)^2]
// slots: 0 power spectrum, 2-3 bispectrum, 4 mesh-level adjoint (tables stay cached per slot)
npc_status get_bin_table(npc_ctx* ctx, int n, double box, const npc_kbins& kb, const int16_t** out, int slot = 0);
// twiddle table exp(-2 pi i j / n), j < n, as cplx<T>
npc_status get_twiddles(npc_ctx* ctx, int n, int prec, const void** out);

// ---------------------------------------------------------------------------------------------
// Bispectrum (bispec.cu)
// ---------------------------------------------------------------------------------------------
npc_status run_bispectrum(npc_ctx* ctx, const npc_mesh_spec& m, const npc_kbins& kb, int scoc_mask, int tripo_mask,
                          int shot, int prec, const DevCatalog& d, const DevCatalog* r, double* sc, double* out,
                          int64_t len);
int64_t bispec_counts(const npc_kbins& kb, int64_t* ntri, int64_t* npair);

// Sugiyama TripoSH multipoles B_{l1 l2 L} requested from the bispectrum pipeline (global line of
// sight): output [nmult][nb][nb] estimate, [nmult][nb][nb] shot noise, the mode count of every
// bin, then 8 scalars
constexpr int NPC_SUGI_MAX = 16;
struct SugiReq {
  int nmult;
  int l1[NPC_SUGI_MAX], l2[NPC_SUGI_MAX], L[NPC_SUGI_MAX];
};
npc_status run_bispectrum_sugiyama(npc_ctx* ctx, const npc_mesh_spec& m, const npc_kbins& kb, const SugiReq& req,
                                   int shot, int prec, const DevCatalog& d, const DevCatalog* r, double* sc,
                                   double* out, int64_t len);
npc_status bispec_triangles(const npc_kbins& kb, int32_t* tri, int64_t cap, int64_t* ntri);
// multi-tracer bispectra: tracers 2 and 3 (tracer 1 is the call's catalogue), with their randoms
// (survey geometry) and catalogue scalars
struct CrossReq {
  DevCatalog d[2];
  DevCatalog r[2];
  bool has_r;
  double* sc[2];
};
npc_status run_bispectrum_cross(npc_ctx* ctx, const npc_mesh_spec& m, const npc_kbins& kb, int scoc_mask,
                                int tripo_mask, int prec, const DevCatalog& d, const DevCatalog* r, double* sc1,
                                double* scx, const CrossReq& req, double* out, int64_t len);
