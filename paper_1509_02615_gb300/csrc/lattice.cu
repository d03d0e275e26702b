// Lattice operator storage: one packed weight row per class of nodes whose
// stencils are translates of each other (the optimisation beyond the
// paper's per-node storage of Sec. 3, where every node keeps its own row of
// each differentiation matrix).
//
// On a Cartesian or hexagonal lattice every node away from the walls and
// from the periodic seam sees the same stencil geometry: the same relative
// index offsets j - i (row-major numbering) and the same relative positions
// x_j - x_i.  The augmented systems of Eq. (weights) are then identical, so
// their weights agree up to rounding; nodes of one wall row form a class of
// their own.  A class keeps the weights of its first member, and the stage
// kernel reads (offset, weight) pairs from a table of a few tens of kB that
// stays in L1/L2, instead of ~720 B of per-node operators from HBM.  Nodes
// of classes with fewer than min_members members ("irregular": scattered
// nodes, seams) keep their per-node operators.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "problem.cuh"

namespace rbf {

namespace {

struct KeyHash {
    size_t operator()(const std::vector<int64_t> &k) const {
        uint64_t hsh = 1469598103934665603ull;
        for (int64_t v : k) {
            hsh ^= (uint64_t)v + 0x9e3779b97f4a7c15ull + (hsh << 6) + (hsh >> 2);
            hsh *= 1099511628211ull;
        }
        return (size_t)hsh;
    }
};

// Relative position of j seen from i, periodic in x with the minimum image.
inline double rel_x(double xj, double xi, double period_x) {
    double d = xj - xi;
    if (period_x > 0.0) {
        if (d > 0.5 * period_x) d -= period_x;
        else if (d < -0.5 * period_x) d += period_x;
    }
    return d;
}

}  // namespace

// Classes of translated stencils.  The key of node i is its stencil's
// relative index offsets and its relative positions quantised to h / 2^20;
// returns the class of every node (-1: irregular) and the class count.
// Classes are numbered in the order of their first member.
int32_t lattice_classes(const int32_t *idx, const double *x, const double *z, int64_t n_prog, int n,
                        double period_x, double h, int min_members, int32_t *cls) {
    const double q = 1048576.0 / h;
    std::unordered_map<std::vector<int64_t>, int32_t, KeyHash> key_of;
    key_of.reserve((size_t)std::min<int64_t>(n_prog, 1 << 20));
    std::vector<int32_t> raw(n_prog);
    std::vector<int64_t> count;
    std::vector<int64_t> key(3 * (size_t)n);
    for (int64_t i = 0; i < n_prog; ++i) {
        const int32_t *s = idx + i * n;
        for (int k = 0; k < n; ++k) {
            const int64_t j = s[k];
            key[3 * k] = j - i;
            key[3 * k + 1] = (int64_t)std::llround(rel_x(x[j], x[i], period_x) * q);
            key[3 * k + 2] = (int64_t)std::llround((z[j] - z[i]) * q);
        }
        auto it = key_of.find(key);
        if (it == key_of.end()) {
            it = key_of.emplace(key, (int32_t)count.size()).first;
            count.push_back(0);
        }
        raw[i] = it->second;
        ++count[it->second];
    }
    // keep the classes with enough members, renumbered in first-member order
    std::vector<int32_t> renum(count.size(), -1);
    int32_t n_cls = 0;
    for (int64_t i = 0; i < n_prog; ++i) {
        const int32_t r = raw[i];
        if (count[r] >= min_members && renum[r] < 0) renum[r] = n_cls++;
        cls[i] = count[r] >= min_members ? renum[r] : -1;
    }
    return n_cls;
}

// Builds the class table for the current packing (pb.G, pb.SLQ, pb.V,
// pb.diff): lw = T [4][n_cls][SLQ][G][V] (packed operators of the class's
// first member, combined as `comb`), loff = int32 [n_cls][SLQ][G][V]
// (relative index of every slot; padding slots point at the node itself
// with zero weight).  The class ids are computed once.
void pack_lattice(Problem &pb, const std::vector<double> &comb, int nops) {
    Problem::Lattice &L = pb.lat;
    if (!L.classified) {
        std::vector<int32_t> idx((size_t)pb.n_prog * pb.n);
        std::vector<double> x(pb.n_all), z(pb.n_all);
        RBF_CUDA(cudaMemcpyAsync(idx.data(), pb.idx.p, idx.size() * 4, cudaMemcpyDeviceToHost, pb.st));
        RBF_CUDA(cudaMemcpyAsync(x.data(), pb.x.p, x.size() * 8, cudaMemcpyDeviceToHost, pb.st));
        RBF_CUDA(cudaMemcpyAsync(z.data(), pb.z.p, z.size() * 8, cudaMemcpyDeviceToHost, pb.st));
        RBF_CUDA(cudaStreamSynchronize(pb.st));
        // quantum of the position keys: the smallest nearest-neighbour distance
        double hq = INFINITY;
        for (int64_t i = 0; i < pb.n_prog && pb.n > 1; ++i) {
            const int64_t j = idx[(size_t)i * pb.n + 1];
            const double d = std::hypot(rel_x(x[j], x[i], pb.period_x), z[j] - z[i]);
            if (d > 0.0) hq = std::min(hq, d);
        }
        if (!std::isfinite(hq)) hq = 1.0;
        L.cls_host.assign(pb.n_prog, -1);
        L.n_cls = lattice_classes(idx.data(), x.data(), z.data(), pb.n_prog, pb.n, pb.period_x, hq, L.min_members,
                                  L.cls_host.data());
        L.rep.assign(L.n_cls, -1);
        L.class_nodes = 0;
        for (int64_t i = 0; i < pb.n_prog; ++i) {
            const int32_t c = L.cls_host[i];
            if (c < 0) continue;
            ++L.class_nodes;
            if (L.rep[c] < 0) L.rep[c] = i;
        }
        L.rep_idx.resize((size_t)L.n_cls * pb.n);
        for (int32_t c = 0; c < L.n_cls; ++c)
            for (int k = 0; k < pb.n; ++k) L.rep_idx[(size_t)c * pb.n + k] = idx[(size_t)L.rep[c] * pb.n + k];
        L.rep_w.resize((size_t)nops * L.n_cls * pb.n);
        for (int o = 0; o < nops; ++o)
            for (int32_t c = 0; c < L.n_cls; ++c)
                RBF_CUDA(cudaMemcpyAsync(L.rep_w.data() + ((size_t)o * L.n_cls + c) * pb.n,
                                         pb.w64.p + ((size_t)o * pb.n_prog + L.rep[c]) * pb.n, pb.n * 8,
                                         cudaMemcpyDeviceToHost, pb.st));
        RBF_CUDA(cudaStreamSynchronize(pb.st));
        L.cls.alloc(pb.n_prog);
        RBF_CUDA(cudaMemcpyAsync(L.cls.p, L.cls_host.data(), pb.n_prog * 4, cudaMemcpyHostToDevice, pb.st));
        L.classified = true;
    }
    const int per = pb.SLQ * pb.G * pb.V;
    std::vector<int32_t> off((size_t)L.n_cls * per, 0);
    std::vector<double> w((size_t)4 * L.n_cls * per, 0.0);
    for (int32_t c = 0; c < L.n_cls; ++c) {
        const int64_t i = L.rep[c];
        for (int t = 0; t < per; ++t) {
            // slot t = (q G + g) V + v of the per-node packing, stored at [q][g][v]
            const int v = t % pb.V, gq = t / pb.V;
            const int g = gq % pb.G, qq = gq / pb.G;
            const size_t dst = (((size_t)c * pb.SLQ + qq) * pb.G + g) * pb.V + v;
            if (t >= pb.n_slots) continue;   // padding: self, weight 0
            const int k = t + pb.diff;
            off[dst] = (int32_t)(L.rep_idx[(size_t)c * pb.n + k] - i);
            for (int p = 0; p < 4; ++p) {
                double val = 0.0;
                for (int o = 0; o < nops; ++o) {
                    const double cf = comb[p * nops + o];
                    if (cf != 0.0) val += cf * L.rep_w[((size_t)o * L.n_cls + c) * pb.n + k];
                }
                w[(size_t)p * L.n_cls * per + dst] = val;
            }
        }
    }
    L.loff.alloc(std::max<size_t>(off.size(), 1));
    RBF_CUDA(cudaMemcpyAsync(L.loff.p, off.data(), off.size() * 4, cudaMemcpyHostToDevice, pb.st));
    L.lw.alloc(std::max<size_t>(w.size(), 1) * pb.tsize());
    if (pb.precision == 64) {
        RBF_CUDA(cudaMemcpyAsync(L.lw.p, w.data(), w.size() * 8, cudaMemcpyHostToDevice, pb.st));
    } else {
        std::vector<float> wf(w.begin(), w.end());
        RBF_CUDA(cudaMemcpyAsync(L.lw.p, wf.data(), wf.size() * 4, cudaMemcpyHostToDevice, pb.st));
    }
    RBF_CUDA(cudaStreamSynchronize(pb.st));
}

}  // namespace rbf

extern "C" int rbf_lattice_classes(const int32_t *idx, const double *x, const double *z, int64_t n_prog,
                                   int64_t n_all, int32_t n_sten, double period_x, double h, int32_t min_members,
                                   int32_t *cls, int32_t *n_classes) {
    return rbf::guarded([&] {
        RBF_REQUIRE(idx && x && z && cls && n_classes, "null argument");
        RBF_REQUIRE(n_prog >= 1 && n_all >= n_prog && n_all < ((int64_t)1 << 31), "node counts out of range");
        RBF_REQUIRE(n_sten >= 1, "stencil size must be >= 1");
        RBF_REQUIRE(h > 0.0 && std::isfinite(h), "h must be positive");
        RBF_REQUIRE(min_members >= 1, "min_members must be >= 1");
        RBF_REQUIRE(period_x >= 0.0 && std::isfinite(period_x), "period_x must be >= 0");
        for (int64_t e = 0; e < n_prog * n_sten; ++e)
            RBF_REQUIRE(idx[e] >= 0 && idx[e] < n_all, "idx[%lld] = %d out of range", (long long)e, idx[e]);
        for (int64_t j = 0; j < n_all; ++j)
            RBF_REQUIRE(std::isfinite(x[j]) && std::isfinite(z[j]), "non-finite coordinate at %lld", (long long)j);
        *n_classes = rbf::lattice_classes(idx, x, z, n_prog, n_sten, period_x, h, min_members, cls);
    });
}
