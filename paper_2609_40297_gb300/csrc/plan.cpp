// Tree check and level plan on the host (Sec. III-B ancestor sets, Sec. IV-C depth levels).
//
// The plan orders nodes by depth level L_d (nodes of one level are independent); inside a level,
// internal nodes (those with children, whose depth buffer descendants will read) come first so
// that the render pass covers a prefix. Each node gets its ancestor list A(n), parent first (the
// parent observes most of what a child sees, so the ancestor test usually exits at the first
// entry), its position quantised to Q16 voxel units, and an arena slot for its depth buffer
// (leaves get none).
#include <cmath>

#include "mig_impl.h"

namespace mig {

mig_status tree_check(int n, const int32_t *parent, int32_t *depth, int32_t *max_depth) {
    if (n < 0) return fail(MIG_EINVAL, "tree: negative node count");
    if (n > 0 && !parent) return fail(MIG_EINVAL, "tree: parent array is NULL");
    int roots = 0;
    for (int i = 0; i < n; ++i) {
        const int p = parent[i];
        if (p == -1) {
            roots++;
        } else if (p < 0 || p >= n || p == i) {
            return fail(MIG_EINVAL, "tree: node " + std::to_string(i) + " has an invalid parent " + std::to_string(p));
        }
    }
    if (n > 0 && roots != 1) return fail(MIG_EINVAL, "tree: expected exactly one root, found " + std::to_string(roots));
    // depth by memoised walks; a walk longer than MIG_MAX_DEPTH means a cycle or a too-deep tree
    std::vector<int32_t> d(n, -1);
    std::vector<int32_t> stack;
    int md = 0;
    for (int i = 0; i < n; ++i) {
        int q = i;
        stack.clear();
        while (q >= 0 && d[q] < 0) {
            stack.push_back(q);
            if ((int)stack.size() > MIG_MAX_DEPTH + 1)
                return fail(MIG_EINVAL, "tree: cycle or depth above " + std::to_string(MIG_MAX_DEPTH));
            q = parent[q];
        }
        int base = (q < 0) ? -1 : d[q];
        for (int s = (int)stack.size() - 1; s >= 0; --s) d[stack[s]] = ++base;
        if (base > MIG_MAX_DEPTH) return fail(MIG_EINVAL, "tree: depth above " + std::to_string(MIG_MAX_DEPTH));
        if (base > md) md = base;
    }
    if (depth)
        for (int i = 0; i < n; ++i) depth[i] = d[i];
    if (max_depth) *max_depth = (n > 0) ? md : -1;
    return MIG_OK;
}

mig_status plan_build(int n, const int32_t *parent, const float *pos, const float origin[3], float voxel,
                      const int dims[3], HostPlan &p) {
    p.n = n;
    p.depth.assign(n, 0);
    int md = -1;
    mig_status st = tree_check(n, parent, p.depth.data(), &md);
    if (st != MIG_OK) return st;
    if (n > 0 && !pos) return fail(MIG_EINVAL, "tree: position array is NULL");
    p.max_depth = md;
    const int L = md + 1;
    std::vector<uint8_t> has_child(n, 0);
    for (int i = 0; i < n; ++i)
        if (parent[i] >= 0) has_child[parent[i]] = 1;
    // level CSR, internal nodes first inside each level (stable by node id)
    std::vector<int32_t> cnt(L, 0), cint(L, 0);
    for (int i = 0; i < n; ++i) {
        cnt[p.depth[i]]++;
        if (has_child[i]) cint[p.depth[i]]++;
    }
    p.level_off.assign(L + 1, 0);
    p.level_int.assign(L, 0);
    for (int d = 0; d < L; ++d) {
        p.level_off[d + 1] = p.level_off[d] + cnt[d];
        p.level_int[d] = cint[d];
    }
    p.level_nodes.assign(n, 0);
    std::vector<int32_t> put_int(L), put_leaf(L);
    for (int d = 0; d < L; ++d) {
        put_int[d] = p.level_off[d];
        put_leaf[d] = p.level_off[d] + cint[d];
    }
    for (int i = 0; i < n; ++i) {
        const int d = p.depth[i];
        if (has_child[i]) p.level_nodes[put_int[d]++] = i;
        else p.level_nodes[put_leaf[d]++] = i;
    }
    // ancestors, parent first
    p.anc_off.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) p.anc_off[i + 1] = p.anc_off[i] + p.depth[i];
    p.total_anc = p.anc_off[n];
    p.anc.assign(p.total_anc, 0);
    for (int i = 0; i < n; ++i) {
        int w = p.anc_off[i];
        for (int q = parent[i]; q >= 0; q = parent[q]) p.anc[w++] = q;
    }
    // quantised positions (Q16 voxel units, round half to even) and arena slots
    p.node.assign((size_t)n * 4, 0);
    int slot = 0;
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            const double q = (((double)pos[3 * (size_t)i + a] - (double)origin[a]) / (double)voxel) * 65536.0;
            if (!(q > -1.0 && q < (double)dims[a] * 65536.0))
                return fail(MIG_EINVAL, "tree: node " + std::to_string(i) + " lies outside the grid");
            const int64_t v = std::llrint(q);
            if (v < 0 || v >= (int64_t)dims[a] * kOneQ16)
                return fail(MIG_EINVAL, "tree: node " + std::to_string(i) + " lies outside the grid");
            p.node[(size_t)i * 4 + a] = (int32_t)v;
        }
        p.node[(size_t)i * 4 + 3] = has_child[i] ? slot++ : -1;
    }
    p.n_internal = slot;
    return MIG_OK;
}

}  // namespace mig
