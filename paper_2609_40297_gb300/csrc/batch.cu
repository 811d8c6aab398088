// Batched evaluation of many independent trees (placeholder: sequential per-tree evaluation).
#include "mig_impl.h"

struct mig_ctx::Batch {};

extern "C" void mig_batch_release(mig_ctx *ctx) {
    delete ctx->batch;
    ctx->batch = nullptr;
}

extern "C" mig_status mig_tree_eval_batch(mig_ctx *ctx, int n_trees, const mig_tree_desc *trees) {
    if (!ctx || (n_trees > 0 && !trees)) return mig::fail(MIG_EINVAL, "tree_eval_batch: NULL argument");
    for (int t = 0; t < n_trees; ++t) {
        mig_eval_opts o{};
        o.mode = trees[t].mode;
        mig_status st = mig_tree_eval_ex(trees[t].map, trees[t].n_nodes, trees[t].parent, trees[t].pos_m,
                                         &trees[t].sensor, &o, trees[t].abs_gain, trees[t].marg_gain, trees[t].best_yaw);
        if (st != MIG_OK) return st;
    }
    return MIG_OK;
}

extern "C" mig_status mig_batch_set_tiles(mig_ctx *ctx, const mig_tile_config *cfg) {
    if (!ctx || !cfg) return mig::fail(MIG_EINVAL, "batch_set_tiles: NULL argument");
    if (cfg->tile_w < 1 || cfg->tile_h < 1 || cfg->tile_w * cfg->tile_h > 4096 || (cfg->tile_w * cfg->tile_h) % 32 != 0 ||
        cfg->ctas_per_sm < 1 || cfg->ctas_per_sm > 32)
        return mig::fail(MIG_EINVAL, "batch_set_tiles: a tile holds a multiple of 32 rays, at most 4096");
    ctx->tiles = *cfg;
    return MIG_OK;
}

extern "C" mig_status mig_batch_get_tiles(mig_ctx *ctx, mig_tile_config *cfg) {
    if (!ctx || !cfg) return mig::fail(MIG_EINVAL, "batch_get_tiles: NULL argument");
    *cfg = ctx->tiles;
    return MIG_OK;
}
