// Bounding-volume hierarchy over a mesh's faces for the labeller (a replacement for the linear
// nearest-triangle search the paper names as the cost of mesh ray tracing, Sec. 1). Built once on
// the host when the mesh is created: top-down, binned surface-area heuristic (16 bins per axis
// over the face centroids), leaves of up to 8 faces, depth at most kBvhMaxDepth.
//
// Device layout: two-wide nodes of 64 bytes holding both children's boxes, so one load tests two
// boxes: float4 a = (L.lo.xyz, L.hi.x), b = (L.hi.yz, R.lo.xy), c = (R.lo.z, R.hi.xyz), and int4
// d = (left, right, left count, right count); a child >= 0 is an inner node, a child < 0 a leaf
// holding faces bvh_tri[-(child + 1) ..][0 .. count). Boxes are computed in double from the
// float32 vertices and padded outward (1e-6 relative plus a floor, rounded away from the box), so
// a box contains every point the float64 Moeller-Trumbore test can accept on its faces and the
// float32 slab test never drops a face the float64 test would hit.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ddf_internal.cuh"

namespace ddf {
namespace {

struct Box {
    double lo[3] = {INFINITY, INFINITY, INFINITY};
    double hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    void grow(const Box& b) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], b.lo[a]);
            hi[a] = std::max(hi[a], b.hi[a]);
        }
    }
    void grow(const double p[3]) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], p[a]);
            hi[a] = std::max(hi[a], p[a]);
        }
    }
    double area() const {
        const double x = hi[0] - lo[0], y = hi[1] - lo[1], z = hi[2] - lo[2];
        if (!(x >= 0) || !(y >= 0) || !(z >= 0)) return 0.0;
        return 2.0 * (x * y + y * z + z * x);
    }
};

struct Child {
    int ref = -1;     // inner node index, or -(first + 1) for a leaf
    int count = 0;    // faces of a leaf
    Box box;
};

struct HostNode {
    Child c[2];
};

constexpr int kBins = 16;
constexpr int kLeafMax = 8;

struct Builder {
    std::vector<Box> tbox;
    std::vector<double> cen;   // 3 per face
    std::vector<int32_t> idx;
    std::vector<HostNode> nodes;
    int max_depth_seen = 0;

    Child leaf(int b, int e, const Box& box) {
        Child c;
        c.ref = -(b + 1);
        c.count = e - b;
        c.box = box;
        return c;
    }

    Child build(int b, int e, int depth) {
        Box box, cbox;
        for (int i = b; i < e; ++i) {
            box.grow(tbox[idx[i]]);
            cbox.grow(&cen[3 * (size_t)idx[i]]);
        }
        max_depth_seen = std::max(max_depth_seen, depth);
        const int n = e - b;
        if (n <= 2 || depth >= kBvhMaxDepth) return leaf(b, e, box);
        // binned SAH over the three axes
        double best_cost = INFINITY;
        int best_axis = -1, best_split = 0;
        for (int a = 0; a < 3; ++a) {
            const double ext = cbox.hi[a] - cbox.lo[a];
            if (!(ext > 0)) continue;
            Box bb[kBins];
            int cnt[kBins] = {0};
            for (int i = b; i < e; ++i) {
                int k = (int)(kBins * (cen[3 * (size_t)idx[i] + a] - cbox.lo[a]) / ext);
                k = std::min(kBins - 1, std::max(0, k));
                bb[k].grow(tbox[idx[i]]);
                cnt[k]++;
            }
            Box right[kBins];
            int rc[kBins];
            Box acc;
            int an = 0;
            for (int k = kBins - 1; k >= 1; --k) {
                acc.grow(bb[k]);
                an += cnt[k];
                right[k] = acc;
                rc[k] = an;
            }
            Box left;
            int ln = 0;
            for (int s = 1; s < kBins; ++s) {
                left.grow(bb[s - 1]);
                ln += cnt[s - 1];
                if (ln == 0 || rc[s] == 0) continue;
                const double cost = left.area() * ln + right[s].area() * rc[s];
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = a;
                    best_split = s;
                }
            }
        }
        const double parent = box.area();
        int mid;
        if (best_axis < 0) {
            // coincident centroids: a leaf if it fits, else an arbitrary even split
            if (n <= kLeafMax) return leaf(b, e, box);
            mid = b + n / 2;
        } else {
            // leaf cost n (one test per face) against one traversal step plus the children's
            // expected tests
            const double split_cost = 1.0 + (parent > 0 ? best_cost / parent : (double)n);
            if (n <= kLeafMax && (double)n <= split_cost) return leaf(b, e, box);
            const double ext = cbox.hi[best_axis] - cbox.lo[best_axis];
            const double lo = cbox.lo[best_axis];
            int* first = idx.data() + b;
            int* pm = std::stable_partition(first, idx.data() + e, [&](int t) {
                int k = (int)(kBins * (cen[3 * (size_t)t + best_axis] - lo) / ext);
                k = std::min(kBins - 1, std::max(0, k));
                return k < best_split;
            });
            mid = (int)(pm - idx.data());
            if (mid == b || mid == e) mid = b + n / 2;
        }
        const int slot = (int)nodes.size();
        nodes.emplace_back();
        Child l = build(b, mid, depth + 1);
        Child r = build(mid, e, depth + 1);
        nodes[slot].c[0] = l;
        nodes[slot].c[1] = r;
        Child me;
        me.ref = slot;
        me.box = box;
        return me;
    }
};

// The padded float32 box of a double box.
void pad_box(const Box& b, float lo[3], float hi[3]) {
    for (int a = 0; a < 3; ++a) {
        if (!(b.hi[a] >= b.lo[a])) {   // empty: a box no ray meets
            lo[a] = 1.f;
            hi[a] = -1.f;
            continue;
        }
        const double pad = 1e-6 * (fabs(b.lo[a]) + fabs(b.hi[a]) + (b.hi[a] - b.lo[a])) + 1e-9;
        lo[a] = nextafterf((float)(b.lo[a] - pad), -INFINITY);
        hi[a] = nextafterf((float)(b.hi[a] + pad), INFINITY);
    }
}

}  // namespace

// The device image of the hierarchy of a mesh given on the host: 4 float4 per node (see the top of
// this file), the face order, and the depth. No device call.
void bvh_build_host(const float* hv, const int32_t* ht, int64_t nt, std::vector<float4>& dev,
                    std::vector<int32_t>& order, int* depth) {
    Builder B;
    B.tbox.resize(nt);
    B.cen.resize(3 * nt);
    B.idx.resize(nt);
    for (int64_t k = 0; k < nt; ++k) {
        Box bx;
        double c[3] = {0, 0, 0};
        for (int j = 0; j < 3; ++j) {
            double p[3];
            for (int a = 0; a < 3; ++a) {
                p[a] = hv[3 * (int64_t)ht[3 * k + j] + a];
                c[a] += p[a] / 3.0;
            }
            bx.grow(p);
        }
        B.tbox[k] = bx;
        for (int a = 0; a < 3; ++a) B.cen[3 * k + a] = c[a];
        B.idx[k] = (int32_t)k;
    }
    // the root is always an inner node, in slot 0 (build() allocates a node before its children);
    // a mesh that fits one leaf gets a root with that leaf and an empty second child
    const Child root = B.build(0, (int)nt, 0);
    if (root.ref < 0) {
        B.nodes.emplace_back();
        B.nodes[0].c[0] = root;
        B.nodes[0].c[1].ref = -1;
        B.nodes[0].c[1].count = 0;
    }
    const int64_t nn = (int64_t)B.nodes.size();
    dev.assign(4 * nn, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int64_t i = 0; i < nn; ++i) {
        float lo[2][3], hi[2][3];
        int ref[2], cnt[2];
        for (int s = 0; s < 2; ++s) {
            const Child& c = B.nodes[i].c[s];
            pad_box(c.box, lo[s], hi[s]);
            ref[s] = c.ref;
            cnt[s] = c.ref < 0 ? c.count : 0;
        }
        dev[4 * i + 0] = make_float4(lo[0][0], lo[0][1], lo[0][2], hi[0][0]);
        dev[4 * i + 1] = make_float4(hi[0][1], hi[0][2], lo[1][0], lo[1][1]);
        dev[4 * i + 2] = make_float4(lo[1][2], hi[1][0], hi[1][1], hi[1][2]);
        int4 d = make_int4(ref[0], ref[1], cnt[0], cnt[1]);
        memcpy(&dev[4 * i + 3], &d, sizeof d);
    }
    order = std::move(B.idx);
    *depth = B.max_depth_seen;
}

int bvh_build(ddf_mesh_s* m, const float* hv, const int32_t* ht) {
    const int64_t nt = m->nt;
    std::vector<float4> dev;
    std::vector<int32_t> order;
    int depth = 0;
    bvh_build_host(hv, ht, nt, dev, order, &depth);
    const int64_t nn = (int64_t)dev.size() / 4;
    DDF_CUDA_TRY(cudaMalloc(&m->bvh, sizeof(float4) * 4 * nn));
    DDF_CUDA_TRY(cudaMalloc(&m->bvh_tri, sizeof(int32_t) * std::max<int64_t>(1, nt)));
    DDF_CUDA_TRY(cudaMemcpy(m->bvh, dev.data(), sizeof(float4) * 4 * nn, cudaMemcpyHostToDevice));
    DDF_CUDA_TRY(cudaMemcpy(m->bvh_tri, order.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice));
    m->bvh_nodes = nn;
    m->bvh_depth = depth;
    return DDF_OK;
}

// Host self-check of the hierarchy (no device call): every face in exactly one leaf, every padded
// leaf box holding its faces' vertices, every child box inside its parent's, every inner node
// reached once, depth within kBvhMaxDepth. out: nodes, depth, leaves, largest leaf.
int bvh_check_host(const float* hv, int64_t nv, const int32_t* ht, int64_t nt, int64_t out[4]) {
    std::vector<float4> dev;
    std::vector<int32_t> order;
    int depth = 0;
    bvh_build_host(hv, ht, nt, dev, order, &depth);
    const int64_t nn = (int64_t)dev.size() / 4;
    if ((int64_t)order.size() != nt || depth > kBvhMaxDepth) return fail(DDF_ERR_NUMERIC, "hierarchy shape");
    std::vector<int> seen_face(nt, 0), seen_node(nn, 0);
    int64_t leaves = 0, largest = 0;
    // (node, parent box) pairs; the root's box is unbounded
    struct Item { int node; float lo[3], hi[3]; };
    std::vector<Item> stack;
    Item root{0, {-INFINITY, -INFINITY, -INFINITY}, {INFINITY, INFINITY, INFINITY}};
    stack.push_back(root);
    while (!stack.empty()) {
        const Item it = stack.back();
        stack.pop_back();
        if (it.node < 0 || it.node >= nn || seen_node[it.node]++) return fail(DDF_ERR_NUMERIC, "node %d", it.node);
        const float4 a = dev[4 * it.node], b = dev[4 * it.node + 1], c = dev[4 * it.node + 2];
        int4 d;
        memcpy(&d, &dev[4 * it.node + 3], sizeof d);
        const float lo[2][3] = {{a.x, a.y, a.z}, {b.z, b.w, c.x}};
        const float hi[2][3] = {{a.w, b.x, b.y}, {c.y, c.z, c.w}};
        const int ref[2] = {d.x, d.y}, cnt[2] = {d.z, d.w};
        for (int s = 0; s < 2; ++s) {
            const bool empty = ref[s] < 0 && cnt[s] == 0;
            if (!empty)
                for (int k = 0; k < 3; ++k)
                    if (!(lo[s][k] >= it.lo[k] && hi[s][k] <= it.hi[k] && lo[s][k] <= hi[s][k]))
                        return fail(DDF_ERR_NUMERIC, "child box of node %d outside its parent", it.node);
            if (ref[s] >= 0) {
                Item ch{ref[s], {lo[s][0], lo[s][1], lo[s][2]}, {hi[s][0], hi[s][1], hi[s][2]}};
                stack.push_back(ch);
                continue;
            }
            const int64_t first = -(int64_t)(ref[s] + 1);
            if (cnt[s] < 0 || first + cnt[s] > nt) return fail(DDF_ERR_NUMERIC, "leaf range");
            if (cnt[s] > 0) {
                ++leaves;
                largest = std::max<int64_t>(largest, cnt[s]);
            }
            for (int j = 0; j < cnt[s]; ++j) {
                const int f = order[first + j];
                if (f < 0 || f >= nt || seen_face[f]++) return fail(DDF_ERR_NUMERIC, "face %d placed twice", f);
                for (int v = 0; v < 3; ++v) {
                    const int32_t vi = ht[3 * (int64_t)f + v];
                    if (vi < 0 || vi >= nv) return fail(DDF_ERR_INVALID_ARG, "face %d references vertex %d", f, vi);
                    for (int k = 0; k < 3; ++k) {
                        const float x = hv[3 * (int64_t)vi + k];
                        if (!(x >= lo[s][k] && x <= hi[s][k])) return fail(DDF_ERR_NUMERIC, "face %d outside its leaf", f);
                    }
                }
            }
        }
    }
    for (int64_t f = 0; f < nt; ++f)
        if (seen_face[f] != 1) return fail(DDF_ERR_NUMERIC, "face %lld in no leaf", (long long)f);
    for (int64_t i = 0; i < nn; ++i)
        if (seen_node[i] != 1) return fail(DDF_ERR_NUMERIC, "node %lld unreachable", (long long)i);
    out[0] = nn;
    out[1] = depth;
    out[2] = leaves;
    out[3] = largest;
    return DDF_OK;
}

}  // namespace ddf
