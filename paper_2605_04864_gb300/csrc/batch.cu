// Batched measurements: many mocks of uneven catalogue size and mesh (P_l and the Scoccimarro
// monopole B_0 of each) enqueued as one CUDA graph.
//
// The mocks are spread over B branches (longest-processing-time first, by n^3 log n); each branch
// is a private context with its own stream and workspace and runs its mocks one after another, so
// B measurements run concurrently and fill the GPU even when each mesh alone would not.  With
// NPC_BATCH_GRAPH the first call of a batch shape runs eagerly (which sizes every workspace and
// uploads every per-mock table: bin tables, shell tables and triangle counts are cached per
// measurement slot), then captures the same enqueue sequence into a graph; later calls with the
// same shape replay it with a single cudaGraphLaunch.  A graph is rebuilt whenever a branch's
// workspace has moved since its capture.  npc_batch_tune times the y-pass tile for every mesh size
// in the batch and the number of branches, and keeps the fastest.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "npc_internal.cuh"

struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<uint64_t> gens;   // ws_generation of each branch context at capture
  int launches = 0;             // kernels in the graph
};

namespace {

constexpr int MAX_BRANCHES = 16;

struct Item {
  const npc_batch_item* it;
  int64_t off_p, off_b, len_p, len_b;
  double cost;
  int branch;
  int index;
};

int64_t power_len(const npc_kbins& kb, uint32_t ell_mask) { return npc_power_out_len(&kb, ell_mask, 0); }

int64_t bispec0_len(const npc_kbins& kb) {
  int64_t ntri = 0, npair = 0;
  bispec_counts(kb, &ntri, &npair);
  return 2 * ntri + ntri + kb.nbins + 8;   // B_0, its shot noise, N_T, N_modes, scalars
}

npc_status check_item(npc_ctx* ctx, const npc_batch_item& it, uint32_t ell_mask, int prec, int i) {
  NPC_TRY(check_spec(ctx, &it.mesh));
  NPC_TRY(check_bins(ctx, &it.power_bins));
  NPC_TRY(check_catalog(ctx, &it.data, "data", false));
  if (!it.data.on_device || it.data.n == 0)
    return set_err(ctx, NPC_ERR_INVALID_ARG, "item %d: data must be a non-empty device catalogue", i);
  if (it.mesh.periodic) {
    if (it.randoms.n != 0) return set_err(ctx, NPC_ERR_INVALID_ARG, "item %d: periodic box takes no randoms", i);
  } else {
    NPC_TRY(check_catalog(ctx, &it.randoms, "randoms", true));
    NPC_TRY(check_painted_pair(ctx, &it.data, &it.randoms));
    if (!it.randoms.on_device || it.randoms.n == 0)
      return set_err(ctx, NPC_ERR_INVALID_ARG, "item %d: survey needs a non-empty device random catalogue", i);
  }
  if (prec == NPC_PREC_FP64 && it.mesh.n > 256)
    return set_err(ctx, NPC_ERR_UNSUPPORTED, "item %d: FP64 precision supports n <= 256", i);
  if (it.bispec_bins.nbins > 0) {
    NPC_TRY(check_bins(ctx, &it.bispec_bins));
    if (it.bispec_bins.nbins > 24) return set_err(ctx, NPC_ERR_UNSUPPORTED, "item %d: at most 24 bispectrum bins", i);
    if (it.mesh.n > 512) return set_err(ctx, NPC_ERR_UNSUPPORTED, "item %d: bispectrum supports n <= 512", i);
    const double kf = 2.0 * M_PI / it.mesh.box;
    const double kmax = it.bispec_bins.kmin + it.bispec_bins.nbins * it.bispec_bins.dk;
    if (kmax > 0.25 * kf * it.mesh.n)
      return set_err(ctx, NPC_ERR_UNSUPPORTED, "item %d: largest bispectrum bin edge exceeds k_N/2", i);
  } else if (it.bispec_bins.nbins < 0) {
    return set_err(ctx, NPC_ERR_INVALID_ARG, "item %d: bispectrum nbins < 0", i);
  }
  (void)ell_mask;
  return NPC_OK;
}

npc_status ensure_branches(npc_ctx* ctx, int nb) {
  while ((int)ctx->subs.size() < nb) {
    npc_ctx* c = nullptr;
    const npc_status st = npc_create(&c, ctx->device, nullptr);
    if (st != NPC_OK) return set_err(ctx, st, "cannot create a batch branch context");
    ctx->subs.push_back(c);
  }
  return NPC_OK;
}

DevCatalog dev_of(const npc_catalog& c) {
  DevCatalog d;
  d.pos = c.pos;
  d.w = c.w;
  d.nbar = c.nbar;
  d.n = c.n;
  d.dtype = c.dtype;
  return d;
}

npc_status run_item(npc_ctx* sub, const Item& I, uint32_t ell_mask, int prec, double* out) {
  const npc_batch_item& it = *I.it;
  sub->slot_base = 1 + I.index;
  const DevCatalog d = dev_of(it.data);
  const DevCatalog r = dev_of(it.randoms);
  const DevCatalog* rp = it.mesh.periodic ? nullptr : &r;
  double* sc;
  NPC_TRY(ws_get(sub, "scalars", sizeof(double) * SC_COUNT, (void**)&sc));
  NPC_TRY(launch_catalog_scalars(sub, d, rp, it.mesh.box, sc));
  NPC_TRY(power_core(sub, it.mesh, d, rp, it.power_bins, ell_mask, 0, prec, sc, out + I.off_p));
  if (it.bispec_bins.nbins > 0)
    NPC_TRY(run_bispectrum(sub, it.mesh, it.bispec_bins, 1, 0, 1, prec, d, rp, sc, out + I.off_b, I.len_b));
  return NPC_OK;
}

struct Events {
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[MAX_BRANCHES] = {};
};

npc_status make_events(npc_ctx* ctx, Events& ev, int nb) {
  NPC_CUDA(ctx, cudaEventCreateWithFlags(&ev.fork, cudaEventDisableTiming));
  for (int b = 0; b < nb; ++b) NPC_CUDA(ctx, cudaEventCreateWithFlags(&ev.join[b], cudaEventDisableTiming));
  return NPC_OK;
}

void free_events(Events& ev, int nb) {
  if (ev.fork) cudaEventDestroy(ev.fork);
  for (int b = 0; b < nb; ++b)
    if (ev.join[b]) cudaEventDestroy(ev.join[b]);
}

// fork from `hub` into the branch streams, enqueue every branch's items, join back into `hub`
npc_status enqueue(npc_ctx* ctx, cudaStream_t hub, const std::vector<Item>& items, int nb, uint32_t ell_mask,
                   int prec, double* out, Events& ev) {
  NPC_CUDA(ctx, cudaEventRecord(ev.fork, hub));
  for (int b = 0; b < nb; ++b) NPC_CUDA(ctx, cudaStreamWaitEvent(ctx->subs[b]->stream, ev.fork, 0));
  for (int b = 0; b < nb; ++b) {
    npc_ctx* sub = ctx->subs[b];
    for (const Item& I : items) {
      if (I.branch != b) continue;
      const npc_status st = run_item(sub, I, ell_mask, prec, out);
      if (st != NPC_OK) return set_err(ctx, st, "batch item %d: %s", I.index, sub->last_error.c_str());
    }
    NPC_CUDA(ctx, cudaEventRecord(ev.join[b], sub->stream));
    NPC_CUDA(ctx, cudaStreamWaitEvent(hub, ev.join[b], 0));
  }
  return NPC_OK;
}

std::string batch_key(int nitems, const npc_batch_item* items, uint32_t ell_mask, int prec, int nb, const double* out,
                      bool tc) {
  std::string k;
  k.push_back(tc ? 'T' : 'M');   // triple-product path baked into the captured kernels
  k.append((const char*)items, sizeof(npc_batch_item) * (size_t)nitems);
  k.append((const char*)&ell_mask, sizeof(ell_mask));
  k.append((const char*)&prec, sizeof(prec));
  k.append((const char*)&nb, sizeof(nb));
  k.append((const char*)&out, sizeof(out));
  return k;
}

npc_status plan_items(npc_ctx* ctx, int nitems, const npc_batch_item* items, uint32_t ell_mask, int prec, int nb,
                      std::vector<Item>* plan, int64_t* total) {
  plan->clear();
  int64_t off = 0;
  for (int i = 0; i < nitems; ++i) {
    NPC_TRY(check_item(ctx, items[i], ell_mask, prec, i));
    Item I{};
    I.it = &items[i];
    I.index = i;
    I.len_p = power_len(items[i].power_bins, ell_mask);
    if (I.len_p == 0) return set_err(ctx, NPC_ERR_INVALID_ARG, "ell_mask must use bits 0, 2, 4");
    I.off_p = off;
    off += I.len_p;
    if (items[i].bispec_bins.nbins > 0) {
      I.len_b = bispec0_len(items[i].bispec_bins);
      I.off_b = off;
      off += I.len_b;
    } else {
      I.off_b = -1;
    }
    const double n3 = std::pow((double)items[i].mesh.n, 3);
    I.cost = n3 * std::log2(n3) * (items[i].bispec_bins.nbins > 0 ? 3.0 : 1.0) +
             40.0 * (double)(items[i].data.n + items[i].randoms.n);
    plan->push_back(I);
  }
  // longest processing time first onto the least loaded branch (ties: lowest index)
  std::vector<int> order(plan->size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return (*plan)[a].cost > (*plan)[b].cost; });
  std::vector<double> load(nb, 0.0);
  for (int i : order) {
    const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    (*plan)[i].branch = b;
    load[b] += (*plan)[i].cost;
  }
  *total = off;
  return NPC_OK;
}

cudaStream_t hub_stream(npc_ctx* ctx) {
  if (!ctx->batch_hub && cudaStreamCreateWithFlags(&ctx->batch_hub, cudaStreamNonBlocking) != cudaSuccess)
    ctx->batch_hub = nullptr;
  return ctx->batch_hub;
}

// One batch on ctx: eager, or through a cached graph.
npc_status batch_exec(npc_ctx* ctx, int nitems, const npc_batch_item* items, uint32_t ell_mask, int prec,
                      double* out, bool use_graph, int nb) {
  std::vector<Item> plan;
  int64_t total = 0;
  NPC_TRY(plan_items(ctx, nitems, items, ell_mask, prec, nb, &plan, &total));
  NPC_TRY(ensure_branches(ctx, nb));
  for (int b = 0; b < nb; ++b) {
    ctx->subs[b]->ytx = ctx->ytx;
    ctx->subs[b]->use_tcgen05 = ctx->use_tcgen05;
    ctx->subs[b]->wait_limit = ctx->wait_limit;
  }
  cudaStream_t hub = hub_stream(ctx);
  if (!hub) return set_err(ctx, NPC_ERR_CUDA, "cannot create the batch stream");
  Events ev;
  npc_status st = make_events(ctx, ev, nb);
  if (st != NPC_OK) {
    free_events(ev, nb);
    return st;
  }
  // order the batch after the caller's prior work on ctx->stream, and the caller's later work after it
  cudaEvent_t in_ev = ev.fork;
  NPC_CUDA(ctx, cudaEventRecord(in_ev, ctx->stream));
  NPC_CUDA(ctx, cudaStreamWaitEvent(hub, in_ev, 0));
  int launches0 = 0;
  for (int b = 0; b < nb; ++b) launches0 += ctx->subs[b]->launches;

  const std::string key = batch_key(nitems, items, ell_mask, prec, nb, out, ctx->use_tcgen05);
  auto git = ctx->graphs.find(key);
  bool replay = false;
  if (use_graph && git != ctx->graphs.end()) {
    replay = true;
    for (int b = 0; b < nb; ++b) replay = replay && git->second->gens[b] == ctx->subs[b]->ws_generation;
  }
  if (replay) {
    st = cudaGraphLaunch(git->second->exec, hub) == cudaSuccess ? NPC_OK
                                                                 : set_err(ctx, NPC_ERR_CUDA, "graph launch failed");
  } else {
    st = enqueue(ctx, hub, plan, nb, ell_mask, prec, out, ev);
    // a second eager pass settles every first-use cache (e.g. the triangle counts, computed once
    // per geometry, change the enqueued sequence after the first call)
    if (st == NPC_OK && use_graph) st = enqueue(ctx, hub, plan, nb, ell_mask, prec, out, ev);
    if (st == NPC_OK && use_graph) {
      // capture the same sequence (every workspace and table is now in place)
      if (cudaStreamSynchronize(hub) != cudaSuccess) st = set_err(ctx, NPC_ERR_CUDA, "batch warm-up failed");
      cudaGraph_t graph = nullptr;
      int launches1w = 0;
      for (int b = 0; b < nb; ++b) launches1w += ctx->subs[b]->launches;
      if (st == NPC_OK) {
        for (int b = 0; b < nb; ++b) ctx->subs[b]->capturing = true;
        if (cudaStreamBeginCapture(hub, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
          st = set_err(ctx, NPC_ERR_CUDA, "cannot begin graph capture");
        } else {
          const npc_status est = enqueue(ctx, hub, plan, nb, ell_mask, prec, out, ev);
          const cudaError_t ce = cudaStreamEndCapture(hub, &graph);
          if (est != NPC_OK) st = est;
          else if (ce != cudaSuccess) st = set_err(ctx, NPC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
        }
        for (int b = 0; b < nb; ++b) ctx->subs[b]->capturing = false;
      }
      if (st == NPC_OK && graph) {
        cudaGraphExec_t exec = nullptr;
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
          st = set_err(ctx, NPC_ERR_CUDA, "graph instantiation failed");
        } else {
          BatchGraph* g = git != ctx->graphs.end() ? git->second : new BatchGraph();
          if (g->exec) cudaGraphExecDestroy(g->exec);
          g->exec = exec;
          g->gens.assign(nb, 0);
          for (int b = 0; b < nb; ++b) g->gens[b] = ctx->subs[b]->ws_generation;
          int lc = 0;
          for (int b = 0; b < nb; ++b) lc += ctx->subs[b]->launches;
          g->launches = (lc - launches1w);       // kernels enqueued by the capture
          ctx->graphs[key] = g;
        }
      }
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
    }
  }
  if (st == NPC_OK) {
    cudaEvent_t out_ev = ev.join[0];
    if (cudaEventRecord(out_ev, hub) != cudaSuccess || cudaStreamWaitEvent(ctx->stream, out_ev, 0) != cudaSuccess)
      st = set_err(ctx, NPC_ERR_CUDA, "cannot join the batch stream");
  }
  // events may be destroyed once recorded: CUDA releases them when their work completes
  free_events(ev, nb);
  int launches1 = 0;
  for (int b = 0; b < nb; ++b) launches1 += ctx->subs[b]->launches;
  int kernels = launches1 - launches0;
  if (use_graph) {
    auto g2 = ctx->graphs.find(key);
    if (g2 != ctx->graphs.end()) kernels = g2->second->launches;
  }
  ctx->launches += kernels;
  return st;
}

int default_branches(const npc_ctx* ctx, int nitems) {
  const int b = ctx->batch_branches > 0 ? ctx->batch_branches : 4;
  return std::max(1, std::min({b, nitems, MAX_BRANCHES}));
}

}  // namespace

void destroy_batch_state(npc_ctx* ctx) {
  for (auto& kv : ctx->graphs) {
    if (kv.second->exec) cudaGraphExecDestroy(kv.second->exec);
    delete kv.second;
  }
  ctx->graphs.clear();
  for (npc_ctx* s : ctx->subs) npc_destroy(s);
  ctx->subs.clear();
  if (ctx->batch_hub) cudaStreamDestroy(ctx->batch_hub);
  ctx->batch_hub = nullptr;
}

extern "C" {

int64_t npc_batch_layout(int32_t nitems, const npc_batch_item* items, uint32_t ell_mask, int64_t* offsets) {
  if (nitems < 1 || !items) return 0;
  int64_t off = 0;
  for (int i = 0; i < nitems; ++i) {
    const int64_t lp = power_len(items[i].power_bins, ell_mask);
    if (lp == 0) return 0;
    if (offsets) offsets[2 * i] = off;
    off += lp;
    if (items[i].bispec_bins.nbins > 0) {
      if (items[i].bispec_bins.nbins > 24 || !(items[i].bispec_bins.dk > 0)) return 0;
      if (offsets) offsets[2 * i + 1] = off;
      off += bispec0_len(items[i].bispec_bins);
    } else if (offsets) {
      offsets[2 * i + 1] = -1;
    }
  }
  return off;
}

npc_status npc_batch_run(npc_ctx* ctx, int32_t nitems, const npc_batch_item* items, uint32_t ell_mask,
                         npc_precision prec, double* out_device, int32_t flags) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  begin_call(ctx);
  if (nitems < 1 || !items || !out_device) return set_err(ctx, NPC_ERR_INVALID_ARG, "empty batch or NULL pointer");
  if (prec != NPC_PREC_FP64 && prec != NPC_PREC_MIXED) return set_err(ctx, NPC_ERR_INVALID_ARG, "bad precision");
  if (flags & ~NPC_BATCH_GRAPH) return set_err(ctx, NPC_ERR_INVALID_ARG, "unknown flags");
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));
  NPC_TRY(batch_exec(ctx, nitems, items, ell_mask, prec, out_device, (flags & NPC_BATCH_GRAPH) != 0,
                     default_branches(ctx, nitems)));
  return end_call(ctx);
}

npc_status npc_batch_tune(npc_ctx* ctx, int32_t nitems, const npc_batch_item* items, uint32_t ell_mask,
                          npc_precision prec, double* out_device, int32_t* branches) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  begin_call(ctx);
  if (nitems < 1 || !items || !out_device) return set_err(ctx, NPC_ERR_INVALID_ARG, "empty batch or NULL pointer");
  if (prec != NPC_PREC_FP64 && prec != NPC_PREC_MIXED) return set_err(ctx, NPC_ERR_INVALID_ARG, "bad precision");
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));
  std::vector<Item> plan;
  int64_t total = 0;
  NPC_TRY(plan_items(ctx, nitems, items, ell_mask, prec, 1, &plan, &total));
  // 1. y-pass tile per mesh size (each branch context keeps its own copy of the choice)
  std::vector<int> sizes;
  for (int i = 0; i < nitems; ++i) sizes.push_back(items[i].mesh.n);
  std::sort(sizes.begin(), sizes.end());
  sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
  for (int n : sizes) {
    const int nplanes = std::min(n / 2, 64) * 4;
    NPC_TRY(tune_y_pass(ctx, n, prec, nplanes));
  }
  NPC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  // 2. number of concurrent branches, timed on graph replays
  cudaEvent_t e0, e1;
  NPC_CUDA(ctx, cudaEventCreate(&e0));
  NPC_CUDA(ctx, cudaEventCreate(&e1));
  float best = 1e30f;
  int best_b = 1;
  npc_status st = NPC_OK;
  for (int nb : {1, 2, 4, 8}) {
    if (nb > nitems || nb > MAX_BRANCHES) break;
    st = batch_exec(ctx, nitems, items, ell_mask, prec, out_device, true, nb);   // warm + capture
    if (st == NPC_OK) st = batch_exec(ctx, nitems, items, ell_mask, prec, out_device, true, nb);  // replay
    if (st != NPC_OK) break;
    cudaEventRecord(e0, ctx->stream);
    for (int rep = 0; rep < 2 && st == NPC_OK; ++rep)
      st = batch_exec(ctx, nitems, items, ell_mask, prec, out_device, true, nb);
    cudaEventRecord(e1, ctx->stream);
    if (st != NPC_OK) break;
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < 0.97f * best) {
      best = ms;
      best_b = nb;
    }
  }
  // 3. triple-product path of the bispectra (tcgen05 tiles of 128 rows, or warp-level mma.sync tiles
  //    of 16 rows), timed on graph replays with the chosen branch count
  float best_t = 1e30f;
  bool best_tc = ctx->use_tcgen05;
  for (int opt = 1; opt >= 0 && st == NPC_OK; --opt) {
    ctx->use_tcgen05 = opt != 0;
    st = batch_exec(ctx, nitems, items, ell_mask, prec, out_device, true, best_b);
    if (st == NPC_OK) st = batch_exec(ctx, nitems, items, ell_mask, prec, out_device, true, best_b);
    if (st != NPC_OK) break;
    cudaEventRecord(e0, ctx->stream);
    for (int rep = 0; rep < 2 && st == NPC_OK; ++rep)
      st = batch_exec(ctx, nitems, items, ell_mask, prec, out_device, true, best_b);
    cudaEventRecord(e1, ctx->stream);
    if (st != NPC_OK) break;
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_t) {
      best_t = ms;
      best_tc = opt != 0;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != NPC_OK) return st;
  ctx->use_tcgen05 = best_tc;
  ctx->batch_branches = best_b;
  if (branches) *branches = best_b;
  return end_call(ctx);
}

npc_status npc_tune_transforms(npc_ctx* ctx, int32_t n, npc_precision prec) {
  if (!ctx) return NPC_ERR_INVALID_ARG;
  begin_call(ctx);
  if (prec != NPC_PREC_FP64 && prec != NPC_PREC_MIXED) return set_err(ctx, NPC_ERR_INVALID_ARG, "bad precision");
  NPC_CUDA(ctx, cudaSetDevice(ctx->device));
  NPC_TRY(tune_y_pass(ctx, n, prec, std::min(n / 2, 64) * 4));
  NPC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return end_call(ctx);
}

npc_status npc_batch_set_branches(npc_ctx* ctx, int32_t branches) {
  if (!ctx || branches < 0 || branches > MAX_BRANCHES) return NPC_ERR_INVALID_ARG;
  ctx->batch_branches = branches;
  return NPC_OK;
}

}  // extern "C"
