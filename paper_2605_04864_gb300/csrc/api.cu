// C ABI of libnpc.so: context management, argument validation, device tables and the
// orchestration of the estimator pipelines.  All compute runs in the kernels of catalog.cu,
// power.cu and bispec.cu; the host only validates, allocates workspace and enqueues.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>

#include "npc_internal.cuh"

#define NPC_VERSION "0.1.0"

npc_status set_err(npc_ctx* ctx, npc_status s, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return s;
}

std::string slot_name(const npc_ctx* ctx, const std::string& name) {
  return ctx->slot_base ? name + "#" + std::to_string(ctx->slot_base) : name;
}

npc_status ws_get(npc_ctx* ctx, const char* name, size_t bytes, void** out) {
  Workspace& w = ctx->ws[name];
  if (bytes == 0) bytes = 16;
  if (w.bytes < bytes) {
    if (ctx->capturing)
      return set_err(ctx, NPC_ERR_INVALID_ARG, "workspace '%s' would grow during graph capture", name);
    ctx->ws_generation++;
    // contents cached under this name (tables, triangle counts) do not survive a reallocation
    ctx->host_cache_keys.erase(name);
    if (w.p) {
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return set_err(ctx, NPC_ERR_CUDA, "sync before realloc: %s", cudaGetErrorString(e));
      cudaFree(w.p);
      w.p = nullptr;
      w.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&w.p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      w.p = nullptr;
      return set_err(ctx, NPC_ERR_OOM, "workspace '%s': cannot allocate %zu bytes (%s)", name, bytes,
                     cudaGetErrorString(e));
    }
    w.bytes = bytes;
  }
  *out = w.p;
  return NPC_OK;
}

static bool table_cached(npc_ctx* ctx, const std::string& name0, const std::vector<char>& key, void** out) {
  const std::string name = slot_name(ctx, name0);
  auto it = ctx->host_cache_keys.find(name);
  if (it == ctx->host_cache_keys.end() || it->second != key) return false;
  *out = ctx->ws[name].p;
  return *out != nullptr;
}

npc_status ws_table(npc_ctx* ctx, const std::string& name0, const std::vector<char>& key, const void* data,
                    size_t bytes, void** out) {
  const std::string name = slot_name(ctx, name0);
  void* p;
  NPC_TRY(ws_get(ctx, name.c_str(), bytes, &p));   // (a reallocation drops the cached key)
  auto it = ctx->host_cache_keys.find(name);
  if (it == ctx->host_cache_keys.end() || it->second != key) {
    if (ctx->capturing)
      return set_err(ctx, NPC_ERR_INVALID_ARG, "table '%s' would be uploaded during graph capture", name.c_str());
    NPC_CUDA(ctx, cudaMemcpyAsync(p, data, bytes, cudaMemcpyHostToDevice, ctx->stream));
    NPC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->host_cache_keys[name] = key;
  }
  *out = p;
  return NPC_OK;
}

template <typename V> static void key_push(std::vector<char>& k, const V& v) {
  const char* p = reinterpret_cast<const char*>(&v);
  k.insert(k.end(), p, p + sizeof(V));
}

YNorm ylm_norm_table() {
  YNorm t{};
  for (int l = 0; l <= NPC_LMAX; ++l)
    for (int m = 0; m <= l; ++m) {
      double r = 1.0;  // (l-m)!/(l+m)!
      for (int j = l - m + 1; j <= l + m; ++j) r /= (double)j;
      t.v[l * (l + 1) / 2 + m] = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * r);
      t.f[l * (l + 1) / 2 + m] = (float)t.v[l * (l + 1) / 2 + m];
    }
  return t;
}

npc_status get_twiddles(npc_ctx* ctx, int n, int prec, const void** out) {
  std::vector<char> key;
  key_push(key, n);
  const std::string name = std::string(prec == NPC_PREC_FP64 ? "tw64." : "tw32.") + std::to_string(n);
  void* p;
  if (table_cached(ctx, name, key, &p)) {
    *out = p;
    return NPC_OK;
  }
  if (prec == NPC_PREC_FP64) {
    std::vector<double2> h(n);
    for (int j = 0; j < n; ++j) h[j] = make_double2(std::cos(2.0 * M_PI * j / n), -std::sin(2.0 * M_PI * j / n));
    NPC_TRY(ws_table(ctx, name, key, h.data(), sizeof(double2) * n, &p));
  } else {
    std::vector<float2> h(n);
    for (int j = 0; j < n; ++j)
      h[j] = make_float2((float)std::cos(2.0 * M_PI * j / n), (float)-std::sin(2.0 * M_PI * j / n));
    NPC_TRY(ws_table(ctx, name, key, h.data(), sizeof(float2) * n, &p));
  }
  *out = p;
  return NPC_OK;
}

// bin of every integer |k|^2 = i^2+j^2+l^2 (host, float64, no contraction: -ffp-contract=off)
npc_status get_bin_table(npc_ctx* ctx, int n, double box, const npc_kbins& kb, const int16_t** out, int slot) {
  const std::string name = "bintab" + std::to_string(slot);
  std::vector<char> key;
  key_push(key, n);
  key_push(key, box);
  key_push(key, kb.kmin);
  key_push(key, kb.dk);
  key_push(key, kb.nbins);
  void* cached;
  if (table_cached(ctx, name, key, &cached)) {
    *out = (const int16_t*)cached;
    return NPC_OK;
  }
  const int64_t nmax = 3LL * (n / 2) * (n / 2);
  std::vector<int16_t> h(nmax + 1);
  const double kf = 2.0 * M_PI / box;
  for (int64_t n2 = 0; n2 <= nmax; ++n2) {
    const double kmag = kf * std::sqrt((double)n2);
    const double b = std::floor((kmag - kb.kmin) / kb.dk);
    h[n2] = (n2 > 0 && b >= 0.0 && b < (double)kb.nbins) ? (int16_t)b : (int16_t)-1;
  }
  void* p;
  NPC_TRY(ws_table(ctx, name, key, h.data(), sizeof(int16_t) * h.size(), &p));
  *out = (const int16_t*)p;
  return NPC_OK;
}

// ---------------------------------------------------------------------------------------------
// Validation
// ---------------------------------------------------------------------------------------------
static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
// mesh sizes with compiled transforms: 2^k for 16 <= n <= 1024, and 3 * 2^k for n = 48, 96, 192
static bool mesh_size_ok(int n) { return (is_pow2(n) && n >= 16 && n <= 1024) || n == 48 || n == 96 || n == 192; }

npc_status check_spec(npc_ctx* ctx, const npc_mesh_spec* m) {
  if (!m) return set_err(ctx, NPC_ERR_INVALID_ARG, "mesh spec is NULL");
  if (!mesh_size_ok(m->n))
    return set_err(ctx, NPC_ERR_INVALID_ARG, "mesh n=%d must be a power of two in [16, 1024] or 48, 96, 192", m->n);
  if (!(m->box > 0.0) || !std::isfinite(m->box)) return set_err(ctx, NPC_ERR_INVALID_ARG, "box must be > 0");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(m->origin[a]) || !std::isfinite(m->observer[a]) || !std::isfinite(m->los_dir[a]))
      return set_err(ctx, NPC_ERR_INVALID_ARG, "non-finite origin/observer/los_dir");
  if (m->assign != 2 && m->assign != 3) return set_err(ctx, NPC_ERR_INVALID_ARG, "assign must be 2 (CIC) or 3 (TSC)");
  if (m->interlace != 0 && m->interlace != 1) return set_err(ctx, NPC_ERR_INVALID_ARG, "interlace must be 0 or 1");
  if (m->periodic != 0 && m->periodic != 1) return set_err(ctx, NPC_ERR_INVALID_ARG, "periodic must be 0 or 1");
  if (m->los != 0 && m->los != 1) return set_err(ctx, NPC_ERR_INVALID_ARG, "los must be 0 or 1");
  if (m->los == 1) {
    const double l2 = m->los_dir[0] * m->los_dir[0] + m->los_dir[1] * m->los_dir[1] + m->los_dir[2] * m->los_dir[2];
    if (!(l2 > 0)) return set_err(ctx, NPC_ERR_INVALID_ARG, "los_dir must be non-zero");
  }
  return NPC_OK;
}

npc_status check_catalog(npc_ctx* ctx, const npc_catalog* c, const char* what, bool need_nbar) {
  if (!c) return set_err(ctx, NPC_ERR_INVALID_ARG, "%s catalogue is NULL", what);
  if (c->n < 0) return set_err(ctx, NPC_ERR_INVALID_ARG, "%s: n < 0", what);
  if (c->dtype != 0 && c->dtype != 1) return set_err(ctx, NPC_ERR_INVALID_ARG, "%s: dtype must be 0 or 1", what);
  if (c->on_device != 0 && c->on_device != 1) return set_err(ctx, NPC_ERR_INVALID_ARG, "%s: on_device must be 0/1", what);
  if (c->n > 0 && !c->pos) return set_err(ctx, NPC_ERR_INVALID_ARG, "%s: pos is NULL", what);
  if (c->n > 0 && need_nbar && !c->nbar) return set_err(ctx, NPC_ERR_INVALID_ARG, "%s: nbar is required", what);
  if (c->n >= (int64_t)1 << 31) return set_err(ctx, NPC_ERR_UNSUPPORTED, "%s: more than 2^31-1 objects", what);
  return NPC_OK;
}

// A catalogue and its randoms are sorted into bricks together, with 32-bit offsets into one record
// array: their sizes must sum below 2^31.
npc_status check_painted_pair(npc_ctx* ctx, const npc_catalog* d, const npc_catalog* r) {
  const int64_t tot = d->n + (r ? r->n : 0);
  if (tot >= (int64_t)1 << 31)
    return set_err(ctx, NPC_ERR_UNSUPPORTED, "data + randoms hold %lld objects; painting takes at most 2^31-1",
                   (long long)tot);
  return NPC_OK;
}

npc_status check_bins(npc_ctx* ctx, const npc_kbins* b) {
  if (!b) return set_err(ctx, NPC_ERR_INVALID_ARG, "k-bins are NULL");
  if (!(b->dk > 0.0) || !std::isfinite(b->dk) || !(b->kmin >= 0.0) || !std::isfinite(b->kmin))
    return set_err(ctx, NPC_ERR_INVALID_ARG, "k-bins need dk > 0 and kmin >= 0");
  if (b->nbins < 1 || b->nbins > 4096) return set_err(ctx, NPC_ERR_INVALID_ARG, "nbins must be in [1, 4096]");
  return NPC_OK;
}

// Stage a catalogue on the device (host inputs are copied into context workspace).
npc_status stage_catalog(npc_ctx* ctx, const npc_catalog* c, const char* tag, DevCatalog* out) {
  out->n = c->n;
  out->dtype = c->dtype;
  const size_t es = c->dtype == 1 ? 8 : 4;
  if (c->on_device || c->n == 0) {
    out->pos = c->pos;
    out->w = c->w;
    out->nbar = c->nbar;
    return NPC_OK;
  }
  void *p, *w = nullptr, *nb = nullptr;
  NPC_TRY(ws_get(ctx, (std::string(tag) + ".pos").c_str(), es * 3 * c->n, &p));
  NPC_CUDA(ctx, cudaMemcpyAsync(p, c->pos, es * 3 * c->n, cudaMemcpyHostToDevice, ctx->stream));
  if (c->w) {
    NPC_TRY(ws_get(ctx, (std::string(tag) + ".w").c_str(), es * c->n, &w));
    NPC_CUDA(ctx, cudaMemcpyAsync(w, c->w, es * c->n, cudaMemcpyHostToDevice, ctx->stream));
  }
  if (c->nbar) {
    NPC_TRY(ws_get(ctx, (std::string(tag) + ".nbar").c_str(), es * c->n, &nb));
    NPC_CUDA(ctx, cudaMemcpyAsync(nb, c->nbar, es * c->n, cudaMemcpyHostToDevice, ctx->stream));
  }
  out->pos = p;
  out->w = w;
  out->nbar = nb;
  return NPC_OK;
}

Geom make_geom(const npc_mesh_spec& m) {
  Geom g{};
  g.n = m.n;
  g.h = m.box / m.n;
  for (int a = 0; a < 3; ++a) g.o[a] = m.origin[a] - m.observer[a];
  const double l = std::sqrt(m.los_dir[0] * m.los_dir[0] + m.los_dir[1] * m.los_dir[1] + m.los_dir[2] * m.los_dir[2]);
  for (int a = 0; a < 3; ++a) g.los[a] = l > 0 ? m.los_dir[a] / l : 0.0;
  g.global_los = m.los;
  return g;
}

npc_status stage_begin(npc_ctx* ctx) {
  ctx->stage_names.clear();
  ctx->stage_launches.clear();
  ctx->ev_used = 0;
  ctx->launches_at_mark = ctx->launches;
  if (!ctx->profile) return NPC_OK;
  if (ctx->ev_pool.empty()) {
    cudaEvent_t e;
    NPC_CUDA(ctx, cudaEventCreate(&e));
    ctx->ev_pool.push_back(e);
  }
  NPC_CUDA(ctx, cudaEventRecord(ctx->ev_pool[0], ctx->stream));
  ctx->ev_used = 1;
  return NPC_OK;
}

npc_status stage_mark(npc_ctx* ctx, const char* name) {
  if (!ctx->profile) return NPC_OK;
  if ((int)ctx->ev_pool.size() <= ctx->ev_used) {
    cudaEvent_t e;
    NPC_CUDA(ctx, cudaEventCreate(&e));
    ctx->ev_pool.push_back(e);
  }
  NPC_CUDA(ctx, cudaEventRecord(ctx->ev_pool[ctx->ev_used], ctx->stream));
  ctx->ev_used++;
  ctx->stage_names.push_back(name);
  ctx->stage_launches.push_back(ctx->launches - ctx->launches_at_mark);
  ctx->launches_at_mark = ctx->launches;
  return NPC_OK;
}

void begin_call(npc_ctx* ctx) {
  ctx->launches = 0;
  ctx->bounded_waits = false;
  ctx->contraction_flops = 0.0;
  ctx->contraction_issued_flops = 0.0;
  ctx->contraction_launches = 0;
  ctx->last_error.clear();
  stage_begin(ctx);
}

npc_status end_call(npc_ctx* ctx) {
  ctx->stats.n_kernel_launches = ctx->launches;
  ctx->stats.contraction_flops = ctx->contraction_flops;
  ctx->stats.contraction_launches = ctx->contraction_launches;
  ctx->stats.contraction_issued_flops = ctx->contraction_issued_flops;
  int64_t tot = 0;
  for (auto& kv : ctx->ws) tot += (int64_t)kv.second.bytes;
  ctx->stats.workspace_bytes = tot;
  return NPC_OK;
}

npc_status finish_output(npc_ctx* ctx, const double* dev, double* out, int64_t len, int out_on_device) {
  if (out_on_device) {
    if (dev != out) NPC_CUDA(ctx, cudaMemcpyAsync(out, dev, sizeof(double) * len, cudaMemcpyDeviceToDevice, ctx->stream));
    return NPC_OK;
  }
  NPC_CUDA(ctx, cudaMemcpyAsync(out, dev, sizeof(double) * len, cudaMemcpyDeviceToHost, ctx->stream));
  NPC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->bounded_waits) return check_device_status(ctx);
  return NPC_OK;
}

npc_status check_device_status(npc_ctx* ctx) {
  if (!ctx->dev_status) return NPC_OK;
  int word = 0;
  NPC_CUDA(ctx, cudaMemcpyAsync(&word, ctx->dev_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  NPC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (word == 0) return NPC_OK;
  // tables and counts cached by the failed call may be incomplete: recompute them next time
  ctx->host_cache_keys.clear();
  NPC_CUDA(ctx, cudaMemsetAsync(ctx->dev_status, 0, sizeof(int), ctx->stream));
  NPC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (word == NPC_ERR_NUMERIC)
    return set_err(ctx, NPC_ERR_NUMERIC,
                   "a shell field's largest |value| lies outside [2^-57, 2^63), the range of the f16 tensor-core "
                   "triple products (results of that call are invalid; npc_set_option(\"tcgen05_triple\", 0) "
                   "selects the tf32 mma.sync path)");
  return set_err(ctx, (npc_status)word, "a bounded device-side wait gave up (results of that call are invalid)");
}

// The estimator after validation, staging and the catalogue scalars (device output `dev_out`).
// Field list and pass parameters of one P_l measurement (m >= 0 fields per phase, Table 1).
static PowerPlan make_power_plan(npc_ctx* ctx, const npc_mesh_spec& ms, const npc_kbins& kb, uint32_t ell_mask,
                                 uint32_t modified_mask) {
  const npc_mesh_spec* mesh = &ms;
  const npc_kbins* bins = &kb;
  const int n = mesh->n;
  const int nphase = mesh->interlace ? 2 : 1;
  PowerPlan plan{};
  plan.n = n;
  plan.nphase = nphase;
  plan.ells_mask = (int)ell_mask;
  plan.mod_mask = (int)modified_mask;
  plan.nbins = bins->nbins;
  plan.global_los = mesh->los;
  plan.assign = mesh->assign;
  const Geom g = make_geom(*mesh);
  for (int a = 0; a < 3; ++a) plan.los[a] = g.los[a];
  {
    // rows of the half spectrum that hold no binned mode need not be stored by the y pass (the
    // contraction skips them): a binned mode has k_f |q| < kmin + nbins dk
    const double kf = 2.0 * M_PI / mesh->box, kmax = bins->kmin + bins->nbins * bins->dk;
    const double r2 = (kmax / kf) * (kmax / kf);
    const double full = 3.0 * (n / 2) * (n / 2);
    plan.row_n2max = r2 >= full ? 0 : (int)std::floor(r2) + 1;
    // planes kz > sqrt(row_n2max) hold no binned row: the forward passes stop below them
    if (plan.row_n2max > 0)
      plan.kz_keep = std::min(n / 2, (int)std::floor(std::sqrt((double)plan.row_n2max)) + 1);
  }
  int need = (int)ell_mask | 1;
  if (modified_mask) need |= 1 | 4 | 16;
  FieldList& fl = plan.fl;
  fl.nf = 0;
  int ntr = 0, nr2c = 0;
  auto push = [&](int ph, int l, int m, int part) {
    Comp c;
    c.phase = (int8_t)ph; c.ell = (int8_t)l; c.m = (int8_t)m; c.part = (int8_t)part;
    if (fl.nf < NPC_MAX_FIELDS) fl.f[fl.nf++] = c;   // 2 x 25 at most for l <= 4: always room
  };
  if (mesh->los == 1) {
    for (int ph = 0; ph < nphase; ++ph) push(ph, 0, 0, PART_ONE);
    ntr = 1;
    nr2c = 1;
  } else {
    for (int l = 0; l <= 4; ++l) {
      if (!(need & (1 << l))) continue;
      for (int m = 0; m <= l; ++m) {
        for (int ph = 0; ph < nphase; ++ph) {
          if (l == 0) {
            push(ph, 0, 0, PART_ONE);  // F_0 needs no weighting
            continue;
          }
          push(ph, l, m, PART_RE);
          if (m > 0) push(ph, l, m, PART_IM);
        }
      }
      ntr += l + 1;
      nr2c += 2 * l + 1;
    }
  }
  ctx->stats.n_transforms = ntr;
  ctx->stats.n_r2c_equivalent = nr2c;
  ctx->stats.n_phases = nphase;
  return plan;
}

npc_status power_core(npc_ctx* ctx, const npc_mesh_spec& ms, const DevCatalog& d, const DevCatalog* r,
                      const npc_kbins& kb, uint32_t ell_mask, uint32_t modified_mask, int prec, const double* sc,
                      double* dev_out) {
  const PowerPlan plan = make_power_plan(ctx, ms, kb, ell_mask, modified_mask);
  const int n = ms.n;
  const int nphase = plan.nphase;
  const Geom g = make_geom(ms);
  const size_t rs = prec == NPC_PREC_FP64 ? 8 : 4;
  const size_t ncell = (size_t)n * n * n;
  void *ma, *mb = nullptr, *half;
  NPC_TRY(ws_get(ctx, "mesh.a", rs * ncell, &ma));
  if (nphase == 2) NPC_TRY(ws_get(ctx, "mesh.b", rs * ncell, &mb));
  NPC_TRY(ws_get(ctx, "half", 2 * rs * (size_t)plan.fl.nf * (n / 2) * n * n, &half));
  NPC_TRY(stage_mark(ctx, "alloc"));
  NPC_TRY(launch_paint(ctx, d, r, ms, 1, prec, sc, ma, mb));
  NPC_TRY(stage_mark(ctx, "paint_fold"));
  NPC_TRY(run_forward_transforms(ctx, prec, plan, g, ma, mb, half));
  NPC_TRY(run_power_contract(ctx, prec, plan, ms, kb, half, sc, dev_out));
  return NPC_OK;
}

// Cross multipoles: tracer B's m >= 0 fields and tracer A's F_0 (one field per phase) transformed
// into one half-spectrum buffer, then one contraction of Re[F_0^A F_l^B*].
static npc_status power_cross_core(npc_ctx* ctx, const npc_mesh_spec& ms, const DevCatalog& da,
                                   const DevCatalog* ra, const DevCatalog& db, const DevCatalog* rb,
                                   const npc_kbins& kb, uint32_t ell_mask, int prec, const double* sca,
                                   const double* scb, const double* scx, double* dev_out) {
  PowerPlan plan = make_power_plan(ctx, ms, kb, ell_mask, 0);
  const int nfb = plan.fl.nf;
  PowerPlan plan_a = plan;
  plan_a.fl.nf = 0;
  for (int ph = 0; ph < plan.nphase; ++ph) {
    Comp c;
    c.phase = (int8_t)ph; c.ell = 0; c.m = 0; c.part = PART_ONE;
    plan_a.fl.f[plan_a.fl.nf++] = c;
  }
  if (nfb + plan_a.fl.nf > NPC_MAX_FIELDS) return set_err(ctx, NPC_ERR_UNSUPPORTED, "cross: too many fields");
  const int n = ms.n;
  const Geom g = make_geom(ms);
  const size_t rs = prec == NPC_PREC_FP64 ? 8 : 4;
  const size_t ncell = (size_t)n * n * n;
  const int kzp = plan.kz_keep > 0 ? plan.kz_keep : n / 2;
  const size_t fbytes = 2 * rs * (size_t)kzp * n * n;   // one field's half spectrum (kz < kzp)
  void *ma, *mb = nullptr, *half;
  NPC_TRY(ws_get(ctx, "mesh.a", rs * ncell, &ma));
  if (plan.nphase == 2) NPC_TRY(ws_get(ctx, "mesh.b", rs * ncell, &mb));
  NPC_TRY(ws_get(ctx, "half", fbytes * (size_t)(nfb + plan_a.fl.nf), &half));
  NPC_TRY(stage_mark(ctx, "alloc"));
  NPC_TRY(launch_paint(ctx, db, rb, ms, 1, prec, scb, ma, mb));
  NPC_TRY(stage_mark(ctx, "paint_fold"));
  NPC_TRY(run_forward_transforms(ctx, prec, plan, g, ma, mb, half));
  NPC_TRY(launch_paint(ctx, da, ra, ms, 1, prec, sca, ma, mb));
  NPC_TRY(stage_mark(ctx, "paint_fold_a"));
  NPC_TRY(run_forward_transforms(ctx, prec, plan_a, g, ma, mb, (char*)half + fbytes * nfb));
  for (int f = 0; f < plan_a.fl.nf; ++f) {
    Comp c = plan_a.fl.f[f];
    c.tracer = 1;
    plan.fl.f[plan.fl.nf++] = c;
  }
  plan.cross = 1;
  ctx->stats.n_transforms += 1;
  ctx->stats.n_r2c_equivalent += 1;
  NPC_TRY(run_power_contract(ctx, prec, plan, ms, kb, half, scx, dev_out));
  return NPC_OK;
}

// ---------------------------------------------------------------------------------------------
// Public ABI
// ---------------------------------------------------------------------------------------------
extern "C" {

const char* npc_version(void) { return NPC_VERSION; }

const char* npc_status_string(npc_status s) {
  switch (s) {
    case NPC_OK: return "ok";
    case NPC_ERR_INVALID_ARG: return "invalid argument";
    case NPC_ERR_OOM: return "out of device memory";
    case NPC_ERR_CUDA: return "CUDA error";
    case NPC_ERR_UNSUPPORTED: return "unsupported";
    case NPC_ERR_TIMEOUT: return "device wait timed out";
    case NPC_ERR_NUMERIC: return "degenerate or non-finite normalisation";
  }
  return "unknown status";
}

npc_status npc_create(npc_ctx** out, int device, void* cuda_stream) {
  if (!out) return NPC_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return NPC_ERR_INVALID_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) return NPC_ERR_CUDA;
  npc_ctx* c = new npc_ctx();
  c->device = device;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return NPC_ERR_CUDA;
    }
    c->own_stream = true;
  }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&c->dev_status, 16) != cudaSuccess || cudaMemset(c->dev_status, 0, 16) != cudaSuccess) {
    cudaGetLastError();
    if (c->dev_status) cudaFree(c->dev_status);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return NPC_ERR_OOM;
  }
  *out = c;
  return NPC_OK;
}

npc_status npc_device_status(npc_ctx* ctx) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  // the batch executor's branch contexts first (their kernels run on their own streams)
  for (npc_ctx* sub : ctx->subs) {
    const npc_status st = check_device_status(sub);
    if (st != NPC_OK) return set_err(ctx, st, "%s", sub->last_error.c_str());
  }
  return check_device_status(ctx);
}

npc_status npc_set_wait_limit(npc_ctx* ctx, long long cycles) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  ctx->wait_limit = cycles;
  return NPC_OK;
}

npc_status npc_set_option(npc_ctx* ctx, const char* name, int64_t value) {
  if (!ctx || !name) return NPC_ERR_INVALID_ARG;
  if (std::strcmp(name, "tcgen05_triple") == 0) {
    ctx->use_tcgen05 = value != 0;
    return NPC_OK;
  }
  return set_err(ctx, NPC_ERR_INVALID_ARG, "unknown option '%s'", name);
}

npc_status npc_get_option(npc_ctx* ctx, const char* name, int64_t* value) {
  if (!ctx || !name || !value) return NPC_ERR_INVALID_ARG;
  if (std::strcmp(name, "tcgen05_triple") == 0) {
    *value = ctx->use_tcgen05 ? 1 : 0;
    return NPC_OK;
  }
  if (std::strcmp(name, "batch_branches") == 0) {
    *value = ctx->batch_branches;
    return NPC_OK;
  }
  return set_err(ctx, NPC_ERR_INVALID_ARG, "unknown option '%s'", name);
}

npc_status npc_destroy(npc_ctx* ctx) {
  if (!ctx) return NPC_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  destroy_batch_state(ctx);
  for (auto& kv : ctx->ws)
    if (kv.second.p) cudaFree(kv.second.p);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->dev_status) cudaFree(ctx->dev_status);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return NPC_OK;
}

npc_status npc_last_error(npc_ctx* ctx, char* buf, size_t n) {
  if (!ctx || !buf || n == 0) return NPC_ERR_INVALID_ARG;
  std::strncpy(buf, ctx->last_error.c_str(), n - 1);
  buf[n - 1] = '\0';
  return NPC_OK;
}

npc_status npc_last_stats(npc_ctx* ctx, npc_stats* out) {
  if (!ctx || !out) return NPC_ERR_INVALID_ARG;
  *out = ctx->stats;
  return NPC_OK;
}

npc_status npc_set_profiling(npc_ctx* ctx, int32_t on) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  ctx->profile = on != 0;
  return NPC_OK;
}

npc_status npc_stage_times(npc_ctx* ctx, char* names, double* ms, int32_t* launches, int32_t cap, int32_t* n) {
  if (!ctx || !n) return NPC_ERR_INVALID_ARG;
  *n = 0;
  if (!ctx->profile || ctx->ev_used < 2) return NPC_OK;
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));
  NPC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int ns = std::min<int>((int)ctx->stage_names.size(), cap);
  for (int i = 0; i < ns; ++i) {
    float t = 0.f;
    NPC_CUDA(ctx, cudaEventElapsedTime(&t, ctx->ev_pool[i], ctx->ev_pool[i + 1]));
    if (ms) ms[i] = t;
    if (launches) launches[i] = ctx->stage_launches[i];
    if (names) {
      std::strncpy(names + 32 * i, ctx->stage_names[i].c_str(), 31);
      names[32 * i + 31] = '\0';
    }
  }
  *n = ns;
  return NPC_OK;
}

npc_status npc_catalog_scalars(npc_ctx* ctx, const npc_catalog* data, const npc_catalog* randoms, double box,
                               double* out, int32_t out_on_device) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  begin_call(ctx);
  if (!out) return set_err(ctx, NPC_ERR_INVALID_ARG, "out is NULL");
  NPC_TRY(check_catalog(ctx, data, "data", false));
  if (randoms) NPC_TRY(check_catalog(ctx, randoms, "randoms", true));
  if (!randoms && !(box > 0.0)) return set_err(ctx, NPC_ERR_INVALID_ARG, "periodic scalars need box > 0");
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));
  DevCatalog d, r;
  NPC_TRY(stage_catalog(ctx, data, "data", &d));
  if (randoms) NPC_TRY(stage_catalog(ctx, randoms, "rand", &r));
  double* sc;
  NPC_TRY(ws_get(ctx, "scalars", sizeof(double) * SC_COUNT, (void**)&sc));
  NPC_TRY(launch_catalog_scalars(ctx, d, randoms ? &r : nullptr, box, sc));
  NPC_TRY(finish_output(ctx, sc, out, 8, out_on_device));
  return end_call(ctx);
}

int64_t npc_power_out_len(const npc_kbins* bins, uint32_t ell_mask, uint32_t modified_mask) {
  if (!bins || bins->nbins < 1) return 0;
  if ((ell_mask & ~0x1Fu) || (modified_mask & ~0x70150u) || (ell_mask == 0 && modified_mask == 0)) return 0;
  int rows = 2;
  for (int l = 0; l <= 4; ++l) rows += (ell_mask >> l) & 1;
  for (int l = 4; l <= 8; l += 2) rows += (modified_mask >> l) & 1;
  for (int b = 16; b <= 18; ++b) rows += (modified_mask >> b) & 1;
  return (int64_t)rows * bins->nbins + 8;
}

npc_status npc_power_multipoles(npc_ctx* ctx, const npc_mesh_spec* mesh, const npc_catalog* data,
                                const npc_catalog* randoms, const npc_kbins* bins, uint32_t ell_mask,
                                uint32_t modified_mask, npc_precision prec, double* out, int32_t out_on_device) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  begin_call(ctx);
  NPC_TRY(check_spec(ctx, mesh));
  NPC_TRY(check_bins(ctx, bins));
  if (!out) return set_err(ctx, NPC_ERR_INVALID_ARG, "out is NULL");
  const int64_t out_len = npc_power_out_len(bins, ell_mask, modified_mask);
  if (out_len == 0)
    return set_err(ctx, NPC_ERR_INVALID_ARG, "ell_mask must use bits 0..4 and modified_mask bits 4,6,8,16,17,18");
  if (prec != NPC_PREC_FP64 && prec != NPC_PREC_MIXED) return set_err(ctx, NPC_ERR_INVALID_ARG, "bad precision");
  if (prec == NPC_PREC_FP64 && mesh->n > 256) return set_err(ctx, NPC_ERR_UNSUPPORTED, "FP64 precision supports n <= 256");
  NPC_TRY(check_catalog(ctx, data, "data", false));
  if (mesh->periodic) {
    if (randoms) return set_err(ctx, NPC_ERR_INVALID_ARG, "periodic box takes no randoms");
  } else {
    if (!randoms) return set_err(ctx, NPC_ERR_INVALID_ARG, "survey geometry needs randoms");
    NPC_TRY(check_catalog(ctx, randoms, "randoms", true));
    NPC_TRY(check_painted_pair(ctx, data, randoms));
    if (randoms->n == 0) return set_err(ctx, NPC_ERR_NUMERIC, "empty random catalogue");
  }
  if (data->n == 0) return set_err(ctx, NPC_ERR_NUMERIC, "empty data catalogue (I22 = 0)");
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));

  DevCatalog d, r;
  NPC_TRY(stage_catalog(ctx, data, "data", &d));
  if (randoms) NPC_TRY(stage_catalog(ctx, randoms, "rand", &r));
  double* sc;
  NPC_TRY(ws_get(ctx, "scalars", sizeof(double) * SC_COUNT, (void**)&sc));
  NPC_TRY(stage_mark(ctx, "upload"));
  NPC_TRY(launch_catalog_scalars(ctx, d, randoms ? &r : nullptr, mesh->box, sc));
  NPC_TRY(stage_mark(ctx, "scalars"));
  double* dev_out = out;
  if (!out_on_device) NPC_TRY(ws_get(ctx, "power.out", sizeof(double) * out_len, (void**)&dev_out));
  NPC_TRY(power_core(ctx, *mesh, d, randoms ? &r : nullptr, *bins, ell_mask, modified_mask, prec, sc, dev_out));
  NPC_TRY(finish_output(ctx, dev_out, out, out_len, out_on_device));
  NPC_TRY(stage_mark(ctx, "download"));
  return end_call(ctx);
}

npc_status npc_cross_power_multipoles(npc_ctx* ctx, const npc_mesh_spec* mesh, const npc_catalog* data_a,
                                      const npc_catalog* randoms_a, const npc_catalog* data_b,
                                      const npc_catalog* randoms_b, const npc_kbins* bins, uint32_t ell_mask,
                                      npc_precision prec, double* out, int32_t out_on_device) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  begin_call(ctx);
  NPC_TRY(check_spec(ctx, mesh));
  NPC_TRY(check_bins(ctx, bins));
  if (!out) return set_err(ctx, NPC_ERR_INVALID_ARG, "out is NULL");
  const int64_t out_len = npc_power_out_len(bins, ell_mask, 0);
  if (out_len == 0) return set_err(ctx, NPC_ERR_INVALID_ARG, "ell_mask must use bits 0..4");
  if (prec != NPC_PREC_FP64 && prec != NPC_PREC_MIXED) return set_err(ctx, NPC_ERR_INVALID_ARG, "bad precision");
  if (prec == NPC_PREC_FP64 && mesh->n > 256) return set_err(ctx, NPC_ERR_UNSUPPORTED, "FP64 precision supports n <= 256");
  NPC_TRY(check_catalog(ctx, data_a, "data_a", false));
  NPC_TRY(check_catalog(ctx, data_b, "data_b", false));
  if (mesh->periodic) {
    if (randoms_a || randoms_b) return set_err(ctx, NPC_ERR_INVALID_ARG, "periodic box takes no randoms");
  } else {
    if (!randoms_a || !randoms_b) return set_err(ctx, NPC_ERR_INVALID_ARG, "survey geometry needs both randoms");
    NPC_TRY(check_catalog(ctx, randoms_a, "randoms_a", true));
    NPC_TRY(check_catalog(ctx, randoms_b, "randoms_b", true));
    NPC_TRY(check_painted_pair(ctx, data_a, randoms_a));
    NPC_TRY(check_painted_pair(ctx, data_b, randoms_b));
    if (randoms_a->n == 0 || randoms_b->n == 0) return set_err(ctx, NPC_ERR_NUMERIC, "empty random catalogue");
  }
  if (data_a->n == 0 || data_b->n == 0) return set_err(ctx, NPC_ERR_NUMERIC, "empty data catalogue (I22 = 0)");
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));
  DevCatalog da, ra, db, rb;
  NPC_TRY(stage_catalog(ctx, data_a, "data", &da));
  if (randoms_a) NPC_TRY(stage_catalog(ctx, randoms_a, "rand", &ra));
  NPC_TRY(stage_catalog(ctx, data_b, "data_b", &db));
  if (randoms_b) NPC_TRY(stage_catalog(ctx, randoms_b, "rand_b", &rb));
  double* sc;
  NPC_TRY(ws_get(ctx, "scalars.cross", sizeof(double) * SC_COUNT * 3, (void**)&sc));
  double *sca = sc, *scb = sc + SC_COUNT, *scx = sc + 2 * SC_COUNT;
  NPC_TRY(stage_mark(ctx, "upload"));
  NPC_TRY(launch_catalog_scalars(ctx, da, randoms_a ? &ra : nullptr, mesh->box, sca));
  NPC_TRY(launch_catalog_scalars(ctx, db, randoms_b ? &rb : nullptr, mesh->box, scb));
  NPC_TRY(launch_cross_scalars(ctx, sca, scb, scx));
  NPC_TRY(stage_mark(ctx, "scalars"));
  double* dev_out = out;
  if (!out_on_device) NPC_TRY(ws_get(ctx, "power.out", sizeof(double) * out_len, (void**)&dev_out));
  NPC_TRY(power_cross_core(ctx, *mesh, da, randoms_a ? &ra : nullptr, db, randoms_b ? &rb : nullptr, *bins, ell_mask,
                           prec, sca, scb, scx, dev_out));
  NPC_TRY(finish_output(ctx, dev_out, out, out_len, out_on_device));
  NPC_TRY(stage_mark(ctx, "download"));
  return end_call(ctx);
}

static int64_t bispec_len(const npc_kbins* bins, uint32_t sm, uint32_t tm, int64_t* ntri, int64_t* npair) {
  bispec_counts(*bins, ntri, npair);
  const int ns = ((sm >> 0) & 1) + ((sm >> 1) & 1) + ((sm >> 2) & 1) + ((sm >> 3) & 1);
  const int nt = ((tm >> 0) & 1) + ((tm >> 2) & 1);
  return 2 * ns * (*ntri) + (*ntri) + 2 * nt * (*npair) + bins->nbins + 8;
}

npc_status npc_bispectrum_layout(const npc_kbins* bins, uint32_t scoc_ell_mask, uint32_t tripo_ell_mask,
                                 int64_t* ntri, int64_t* npairs, int64_t* out_len) {
  if (!bins || bins->nbins < 1 || bins->nbins > 24 || !(bins->dk > 0)) return NPC_ERR_INVALID_ARG;
  if ((scoc_ell_mask & ~15u) || (tripo_ell_mask & ~5u) || (scoc_ell_mask | tripo_ell_mask) == 0)
    return NPC_ERR_INVALID_ARG;
  int64_t nt = 0, np = 0;
  const int64_t len = bispec_len(bins, scoc_ell_mask, tripo_ell_mask, &nt, &np);
  if (ntri) *ntri = nt;
  if (npairs) *npairs = np;
  if (out_len) *out_len = len;
  return NPC_OK;
}

npc_status npc_bispectrum_triangles(const npc_kbins* bins, int32_t* tri, int64_t cap, int64_t* ntri) {
  if (!bins || !ntri || bins->nbins < 1 || bins->nbins > 24 || !(bins->dk > 0)) return NPC_ERR_INVALID_ARG;
  return bispec_triangles(*bins, tri, cap, ntri);
}

int64_t npc_bispectrum_sugiyama_len(const npc_kbins* bins, int32_t nmult) {
  if (!bins || bins->nbins < 1 || bins->nbins > 24 || nmult < 1 || nmult > NPC_SUGI_MAX) return -1;
  const int64_t nb = bins->nbins;
  return 2 * (int64_t)nmult * nb * nb + nb + 8;
}

npc_status npc_bispectrum_sugiyama(npc_ctx* ctx, const npc_mesh_spec* mesh, const npc_catalog* data,
                                   const npc_catalog* randoms, const npc_kbins* bins, int32_t nmult,
                                   const int32_t* multipoles, int32_t shot, npc_precision prec, double* out,
                                   int32_t out_on_device) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  begin_call(ctx);
  NPC_TRY(check_spec(ctx, mesh));
  NPC_TRY(check_bins(ctx, bins));
  if (!out) return set_err(ctx, NPC_ERR_INVALID_ARG, "out is NULL");
  if (!multipoles) return set_err(ctx, NPC_ERR_INVALID_ARG, "multipoles is NULL");
  if (nmult < 1 || nmult > NPC_SUGI_MAX) return set_err(ctx, NPC_ERR_INVALID_ARG, "nmult must be 1..%d", NPC_SUGI_MAX);
  if (bins->nbins > 24) return set_err(ctx, NPC_ERR_UNSUPPORTED, "bispectrum supports at most 24 bins");
  SugiReq req{};
  req.nmult = nmult;
  // survey geometry with the line of sight to each grid point: G_L^M for every M (L <= 4)
  const bool endpoint = !mesh->periodic && mesh->los != 1;
  for (int e = 0; e < nmult; ++e) {
    const int l1 = multipoles[3 * e], l2 = multipoles[3 * e + 1], L = multipoles[3 * e + 2];
    // global line of sight: L even (the plane-parallel symmetry about it, Sec. 4.2), so l1 + l2 is
    // even too; endpoint line of sight: l1 + l2 + L even (H_l1l2L != 0), L <= 4
    const bool bad_parity = endpoint ? (((l1 + l2 + L) & 1) || L > 4) : ((L & 1) || ((l1 + l2) & 1));
    if (l1 < 0 || l1 > 4 || l2 < 0 || l2 > 4 || L < std::abs(l1 - l2) || L > l1 + l2 || bad_parity)
      return set_err(ctx, NPC_ERR_INVALID_ARG, "multipole (%d, %d, %d): need l1, l2 <= 4, |l1-l2| <= L <= l1+l2, "
                     "L and l1+l2 even (global line of sight) or l1+l2+L even and L <= 4 (line of sight to each "
                     "grid point)", l1, l2, L);
    req.l1[e] = l1;
    req.l2[e] = l2;
    req.L[e] = L;
  }
  if (prec != NPC_PREC_FP64 && prec != NPC_PREC_MIXED) return set_err(ctx, NPC_ERR_INVALID_ARG, "bad precision");
  if (shot < 0 || shot > 2) return set_err(ctx, NPC_ERR_INVALID_ARG, "shot must be 0, 1 or 2");
  if (mesh->periodic) {
    if (randoms) return set_err(ctx, NPC_ERR_INVALID_ARG, "periodic box takes no randoms");
  } else {
    if (endpoint && shot != 0)
      return set_err(ctx, NPC_ERR_UNSUPPORTED,
                     "TripoSH with the line of sight to each grid point: raw estimates only (shot = 0)");
    if (!randoms) return set_err(ctx, NPC_ERR_INVALID_ARG, "survey geometry needs randoms");
    NPC_TRY(check_catalog(ctx, randoms, "randoms", true));
    NPC_TRY(check_painted_pair(ctx, data, randoms));
    if (randoms->n == 0) return set_err(ctx, NPC_ERR_NUMERIC, "empty random catalogue");
  }
  const double kf = 2.0 * M_PI / mesh->box;
  const double knyq = kf * mesh->n / 2.0;
  const double kmax = bins->kmin + bins->nbins * bins->dk;
  if (kmax > 0.5 * knyq)
    return set_err(ctx, NPC_ERR_UNSUPPORTED, "largest bin edge %.4g exceeds k_N/2 = %.4g (closure would alias)", kmax,
                   0.5 * knyq);
  if (prec == NPC_PREC_FP64 && mesh->n > 256) return set_err(ctx, NPC_ERR_UNSUPPORTED, "FP64 precision supports n <= 256");
  if (mesh->n > 512) return set_err(ctx, NPC_ERR_UNSUPPORTED, "bispectrum supports n <= 512");
  NPC_TRY(check_catalog(ctx, data, "data", false));
  if (data->n == 0) return set_err(ctx, NPC_ERR_NUMERIC, "empty data catalogue (I33 = 0)");
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t out_len = npc_bispectrum_sugiyama_len(bins, nmult);
  ctx->stats.n_transforms = 1;
  ctx->stats.n_r2c_equivalent = 1;
  ctx->stats.n_phases = mesh->interlace ? 2 : 1;
  DevCatalog d, r;
  NPC_TRY(stage_catalog(ctx, data, "data", &d));
  if (randoms) NPC_TRY(stage_catalog(ctx, randoms, "rand", &r));
  double* sc;
  NPC_TRY(ws_get(ctx, "scalars", sizeof(double) * SC_COUNT, (void**)&sc));
  NPC_TRY(stage_mark(ctx, "upload"));
  NPC_TRY(launch_catalog_scalars(ctx, d, randoms ? &r : nullptr, mesh->box, sc));
  NPC_TRY(stage_mark(ctx, "scalars"));
  double* dev_out = out;
  if (!out_on_device) NPC_TRY(ws_get(ctx, "bis.out", sizeof(double) * out_len, (void**)&dev_out));
  NPC_TRY(run_bispectrum_sugiyama(ctx, *mesh, *bins, req, shot, prec, d, randoms ? &r : nullptr, sc, dev_out,
                                  out_len));
  NPC_TRY(finish_output(ctx, dev_out, out, out_len, out_on_device));
  NPC_TRY(stage_mark(ctx, "download"));
  return end_call(ctx);
}

npc_status npc_bispectrum(npc_ctx* ctx, const npc_mesh_spec* mesh, const npc_catalog* data,
                          const npc_catalog* randoms, const npc_kbins* bins, uint32_t scoc_ell_mask,
                          uint32_t tripo_ell_mask, int32_t shot, npc_precision prec, double* out,
                          int32_t out_on_device) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  begin_call(ctx);
  NPC_TRY(check_spec(ctx, mesh));
  NPC_TRY(check_bins(ctx, bins));
  if (!out) return set_err(ctx, NPC_ERR_INVALID_ARG, "out is NULL");
  if (bins->nbins > 24) return set_err(ctx, NPC_ERR_UNSUPPORTED, "bispectrum supports at most 24 bins");
  if ((scoc_ell_mask & ~15u) || (tripo_ell_mask & ~5u) || (scoc_ell_mask | tripo_ell_mask) == 0)
    return set_err(ctx, NPC_ERR_INVALID_ARG, "multipole masks: Scoccimarro bits 0..3, compressed bits 0 and 2");
  if (shot < 0 || shot > 2) return set_err(ctx, NPC_ERR_INVALID_ARG, "shot must be 0, 1 or 2");
  if (prec != NPC_PREC_FP64 && prec != NPC_PREC_MIXED) return set_err(ctx, NPC_ERR_INVALID_ARG, "bad precision");
  const bool mono = (scoc_ell_mask & ~1u) == 0 && (tripo_ell_mask & ~1u) == 0;
  if (mesh->periodic) {
    if (randoms) return set_err(ctx, NPC_ERR_INVALID_ARG, "periodic box takes no randoms");
    if (mesh->los != 1 && !mono)
      return set_err(ctx, NPC_ERR_UNSUPPORTED, "bispectrum: l > 0 in a periodic box needs a global line of sight");
  } else {
    // survey geometry: the monopoles need no line of sight; l = 2 takes the global one (los = 1) or
    // the line of sight to each grid point (Yamamoto X_2), the latter with the analytic shot noise
    if (!mono && mesh->los != 1 && shot == 2)
      return set_err(ctx, NPC_ERR_UNSUPPORTED, "bispectrum: FFT-method shot noise of l = 2 needs a global line of sight");
    if (!randoms) return set_err(ctx, NPC_ERR_INVALID_ARG, "survey geometry needs randoms");
    NPC_TRY(check_catalog(ctx, randoms, "randoms", true));
    NPC_TRY(check_painted_pair(ctx, data, randoms));
    if (randoms->n == 0) return set_err(ctx, NPC_ERR_NUMERIC, "empty random catalogue");
  }
  const double kf = 2.0 * M_PI / mesh->box;
  const double knyq = kf * mesh->n / 2.0;
  const double kmax = bins->kmin + bins->nbins * bins->dk;
  if (kmax > 0.5 * knyq)
    return set_err(ctx, NPC_ERR_UNSUPPORTED, "largest bin edge %.4g exceeds k_N/2 = %.4g (closure would alias)", kmax,
                   0.5 * knyq);
  if (prec == NPC_PREC_FP64 && mesh->n > 256) return set_err(ctx, NPC_ERR_UNSUPPORTED, "FP64 precision supports n <= 256");
  if (mesh->n > 512) return set_err(ctx, NPC_ERR_UNSUPPORTED, "bispectrum supports n <= 512");
  NPC_TRY(check_catalog(ctx, data, "data", false));
  if (data->n == 0) return set_err(ctx, NPC_ERR_NUMERIC, "empty data catalogue (I33 = 0)");
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));
  int64_t ntri = 0, npair = 0;
  const int64_t out_len = bispec_len(bins, scoc_ell_mask, tripo_ell_mask, &ntri, &npair);
  ctx->stats.n_transforms = 1;
  ctx->stats.n_r2c_equivalent = 1;
  ctx->stats.n_phases = mesh->interlace ? 2 : 1;
  DevCatalog d, r;
  NPC_TRY(stage_catalog(ctx, data, "data", &d));
  if (randoms) NPC_TRY(stage_catalog(ctx, randoms, "rand", &r));
  double* sc;
  NPC_TRY(ws_get(ctx, "scalars", sizeof(double) * SC_COUNT, (void**)&sc));
  NPC_TRY(stage_mark(ctx, "upload"));
  NPC_TRY(launch_catalog_scalars(ctx, d, randoms ? &r : nullptr, mesh->box, sc));
  NPC_TRY(stage_mark(ctx, "scalars"));
  double* dev_out = out;
  if (!out_on_device) NPC_TRY(ws_get(ctx, "bis.out", sizeof(double) * out_len, (void**)&dev_out));
  NPC_TRY(run_bispectrum(ctx, *mesh, *bins, (int)scoc_ell_mask, (int)tripo_ell_mask, shot, prec, d,
                         randoms ? &r : nullptr, sc, dev_out, out_len));
  NPC_TRY(finish_output(ctx, dev_out, out, out_len, out_on_device));
  NPC_TRY(stage_mark(ctx, "download"));
  return end_call(ctx);
}

npc_status npc_cross_bispectrum(npc_ctx* ctx, const npc_mesh_spec* mesh, const npc_catalog* data,
                                const npc_catalog* randoms, const npc_kbins* bins, uint32_t scoc_ell_mask,
                                uint32_t tripo_ell_mask, npc_precision prec, double* out, int32_t out_on_device) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  begin_call(ctx);
  NPC_TRY(check_spec(ctx, mesh));
  NPC_TRY(check_bins(ctx, bins));
  if (!out || !data) return set_err(ctx, NPC_ERR_INVALID_ARG, "data and out are required");
  if (bins->nbins > 24) return set_err(ctx, NPC_ERR_UNSUPPORTED, "bispectrum supports at most 24 bins");
  if ((scoc_ell_mask & ~5u) || (tripo_ell_mask & ~5u) || (scoc_ell_mask | tripo_ell_mask) == 0)
    return set_err(ctx, NPC_ERR_INVALID_ARG, "multi-tracer multipole masks must use bits 0 and 2");
  if (prec != NPC_PREC_FP64 && prec != NPC_PREC_MIXED) return set_err(ctx, NPC_ERR_INVALID_ARG, "bad precision");
  if (mesh->los != 1) return set_err(ctx, NPC_ERR_UNSUPPORTED, "multi-tracer bispectra need a global line of sight");
  if (mesh->periodic && randoms) return set_err(ctx, NPC_ERR_INVALID_ARG, "periodic box takes no randoms");
  if (!mesh->periodic && !randoms) return set_err(ctx, NPC_ERR_INVALID_ARG, "survey geometry needs three random catalogues");
  const double kf = 2.0 * M_PI / mesh->box;
  const double kmax = bins->kmin + bins->nbins * bins->dk;
  if (kmax > 0.25 * kf * mesh->n)
    return set_err(ctx, NPC_ERR_UNSUPPORTED, "largest bin edge %.4g exceeds k_N/2 = %.4g (closure would alias)", kmax,
                   0.25 * kf * mesh->n);
  if (prec == NPC_PREC_FP64 && mesh->n > 256) return set_err(ctx, NPC_ERR_UNSUPPORTED, "FP64 precision supports n <= 256");
  if (mesh->n > 512) return set_err(ctx, NPC_ERR_UNSUPPORTED, "bispectrum supports n <= 512");
  static const char* dtag[3] = {"data", "data_b", "data_c"};
  static const char* rtag[3] = {"rand", "rand_b", "rand_c"};
  for (int t = 0; t < 3; ++t) {
    NPC_TRY(check_catalog(ctx, &data[t], dtag[t], false));
    if (data[t].n == 0) return set_err(ctx, NPC_ERR_NUMERIC, "empty data catalogue %d (I33 = 0)", t);
    if (randoms) {
      NPC_TRY(check_catalog(ctx, &randoms[t], rtag[t], true));
      NPC_TRY(check_painted_pair(ctx, &data[t], &randoms[t]));
      if (randoms[t].n == 0) return set_err(ctx, NPC_ERR_NUMERIC, "empty random catalogue %d", t);
    }
  }
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));
  int64_t ntri = 0, npair = 0;
  const int64_t out_len = bispec_len(bins, scoc_ell_mask, tripo_ell_mask, &ntri, &npair);
  DevCatalog d[3], r[3];
  for (int t = 0; t < 3; ++t) {
    NPC_TRY(stage_catalog(ctx, &data[t], dtag[t], &d[t]));
    if (randoms) NPC_TRY(stage_catalog(ctx, &randoms[t], rtag[t], &r[t]));
  }
  double* sc;
  NPC_TRY(ws_get(ctx, "scalars.x3", sizeof(double) * SC_COUNT * 4, (void**)&sc));
  NPC_TRY(stage_mark(ctx, "upload"));
  for (int t = 0; t < 3; ++t)
    NPC_TRY(launch_catalog_scalars(ctx, d[t], randoms ? &r[t] : nullptr, mesh->box, sc + (size_t)t * SC_COUNT));
  double* scx = sc + 3 * SC_COUNT;
  NPC_TRY(launch_cross3_scalars(ctx, sc, sc + SC_COUNT, sc + 2 * SC_COUNT, scx));
  NPC_TRY(stage_mark(ctx, "scalars"));
  CrossReq req{};
  for (int t = 0; t < 2; ++t) {
    req.d[t] = d[1 + t];
    if (randoms) req.r[t] = r[1 + t];
    req.sc[t] = sc + (size_t)(1 + t) * SC_COUNT;
  }
  req.has_r = randoms != nullptr;
  double* dev_out = out;
  if (!out_on_device) NPC_TRY(ws_get(ctx, "bis.out", sizeof(double) * out_len, (void**)&dev_out));
  NPC_TRY(run_bispectrum_cross(ctx, *mesh, *bins, (int)scoc_ell_mask, (int)tripo_ell_mask, prec, d[0],
                               randoms ? &r[0] : nullptr, sc, scx, req, dev_out, out_len));
  NPC_TRY(finish_output(ctx, dev_out, out, out_len, out_on_device));
  NPC_TRY(stage_mark(ctx, "download"));
  return end_call(ctx);
}

}  // extern "C"
