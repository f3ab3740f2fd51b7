// Bispectrum multipoles (placeholder until the shell-field kernels are in place).
#include "npc_internal.cuh"

extern "C" {
npc_status npc_bispectrum(npc_ctx* ctx, const npc_mesh_spec*, const npc_catalog*, const npc_catalog*,
                          const npc_kbins*, uint32_t, uint32_t, int32_t, npc_precision, double*, int32_t) {
  return set_err(ctx, NPC_ERR_UNSUPPORTED, "bispectrum not built yet");
}
npc_status npc_bispectrum_layout(const npc_kbins*, uint32_t, uint32_t, int64_t*, int64_t*, int64_t*) {
  return NPC_ERR_UNSUPPORTED;
}
npc_status npc_bispectrum_triangles(const npc_kbins*, int32_t*, int64_t, int64_t*) { return NPC_ERR_UNSUPPORTED; }
}
