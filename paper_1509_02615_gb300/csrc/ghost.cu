// a4: ghost nodes (Sec. 5.2, Eq. (bcEqn)).
//
// Each wall node gets one ghost outside the domain; the ghost values follow
// from enforcing the boundary conditions at all wall nodes at once:
//     W_G u_G = b - W_I u_I - W_B u_B.
// Setup: the ghosts are split into independent systems (connected components
// of the ghost-coupling graph, e.g. the top and the bottom wall); for every
// component and every distinct boundary-operator pattern the dense W_G block
// is inverted once by Gauss-Jordan elimination with partial pivoting (FP64,
// one launch pair per pivot, all blocks batched).
// Every RK stage: (1) one thread per (field, wall row) forms the residual
// r = b - W_I u_I - W_B u_B from the row's stencil; (2) one warp per
// (class, ghost) forms u_G = W_G^{-1} r from the banded inverse row.  The
// rows of W_G^{-1} decay geometrically along the wall (the wall rows couple
// only nearby ghosts), so each row keeps the entries above 2^-8 eps of its
// largest (eps of the run's precision): the dropped tail is below the
// rounding of the kept sum, and a row reads ~50-100 entries instead of the
// whole component.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>

#include "problem.cuh"
#include "records.cuh"

namespace rbf {

namespace {

// operator of each field's boundary condition: [wall kind][field]
// bottom/top (Sec. 6.3): u_z, w_zz, theta'_z, pi'_z; left/right (Sec. 6.4):
// u_xx, w_x, theta'_x, pi'_x.
const int kBcOps[2][4] = {{RBF_OP_DZ, RBF_OP_DZZ, RBF_OP_DZ, RBF_OP_DZ},
                          {RBF_OP_DXX, RBF_OP_DX, RBF_OP_DX, RBF_OP_DX}};

__global__ void gather_rows(const int32_t *idx, const double *w64, int nops, int64_t n_prog, int n,
                            const int32_t *owner, int64_t ng, int32_t *ridx, double *rw) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ng * n) return;
    int64_t r = t / n;
    int k = (int)(t - r * n);
    int64_t b = owner[r];
    ridx[r * n + k] = idx[b * n + k];
    for (int o = 0; o < nops; ++o) rw[(o * ng + r) * n + k] = w64[((int64_t)o * n_prog + b) * n + k];
}

__global__ void gj_pivot(double *A, double *B, const int *msize, const int64_t *moff, const double *tol,
                         int k, double *colk, int maxm, int *bad) {
    const int mi = blockIdx.x;
    const int m = msize[mi];
    if (k >= m) return;
    double *a = A + moff[mi], *b = B + moff[mi];
    double *col = colk + (int64_t)mi * maxm;
    __shared__ double bv[256];
    __shared__ int bi[256];
    double best = -1.0;
    int besti = k;
    for (int i = k + threadIdx.x; i < m; i += blockDim.x) {
        double v = fabs(a[(int64_t)i * m + k]);
        if (v > best) { best = v; besti = i; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = besti;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double ov = bv[threadIdx.x + s];
            int oi = bi[threadIdx.x + s];
            if (ov > bv[threadIdx.x] || (ov == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = ov;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const int p = bi[0];
    if (!(bv[0] > tol[mi])) {
        if (threadIdx.x == 0) atomicExch(bad, mi + 1);
        return;
    }
    if (p != k) {
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            double t = a[(int64_t)k * m + j];
            a[(int64_t)k * m + j] = a[(int64_t)p * m + j];
            a[(int64_t)p * m + j] = t;
            t = b[(int64_t)k * m + j];
            b[(int64_t)k * m + j] = b[(int64_t)p * m + j];
            b[(int64_t)p * m + j] = t;
        }
    }
    __syncthreads();
    const double inv = 1.0 / a[(int64_t)k * m + k];
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        a[(int64_t)k * m + j] *= inv;
        b[(int64_t)k * m + j] *= inv;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) col[i] = (i == k) ? 0.0 : a[(int64_t)i * m + k];
}

__global__ void gj_eliminate(double *A, double *B, const int *msize, const int64_t *moff, int k,
                             const double *colk, int maxm) {
    const int mi = blockIdx.z;
    const int m = msize[mi];
    const int i = blockIdx.y;
    if (k >= m || i >= m || i == k) return;
    double f = colk[(int64_t)mi * maxm + i];
    if (f == 0.0) return;
    double *a = A + moff[mi], *b = B + moff[mi];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 2 * m; j += gridDim.x * blockDim.x) {
        if (j < m) {
            if (j > k) a[(int64_t)i * m + j] -= f * a[(int64_t)k * m + j];
        } else {
            int jj = j - m;
            b[(int64_t)i * m + jj] -= f * b[(int64_t)k * m + jj];
        }
    }
}

template <class T>
__global__ void to_t(const double *src, T *dst, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (T)src[i];
}

constexpr int kRowLanes = 8;    // lanes per wall row in the residual kernel
constexpr int kRowPf = 16;      // slots per lane held in registers

// r[f][pos(r)] = b_f(r) - sum over the row's non-ghost stencil nodes, all four
// fields at once from one record gather per slot; 8 lanes per row share the
// stencil slots (layout [row][slot]).  U holds node-major records [n_all][4].
template <class T>
__global__ void __launch_bounds__(256) ghost_residual(const T *__restrict__ U, int64_t ng, int64_t rows, int npad,
                                                      const int32_t *__restrict__ gidx, const T *__restrict__ gw,
                                                      const int32_t *__restrict__ owner,
                                                      const unsigned char *__restrict__ tb,
                                                      const int32_t *__restrict__ pos, T *__restrict__ res,
                                                      T cp_tb2, T theta_bar, T gconst) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t r = tid / kRowLanes;
    const int ln = (int)(tid % kRowLanes);
    const bool live = r < rows;
    if (!live) r = rows - 1;
    const int per = npad / kRowLanes;
    // constant operands first: they do not depend on the previous kernel
    int jj[kRowPf];
    T w0[kRowPf], w1[kRowPf], w2[kRowPf], w3[kRowPf];
#pragma unroll
    for (int t = 0; t < kRowPf; ++t) {
        if (t < per) {
            const int64_t o = r * npad + ln + kRowLanes * t;
            jj[t] = __ldg(gidx + o);
            w0[t] = __ldg(gw + o);
            w1[t] = __ldg(gw + ng * npad + o);
            w2[t] = __ldg(gw + 2 * ng * npad + o);
            w3[t] = __ldg(gw + 3 * ng * npad + o);
        }
    }
    grid_dep_wait();
    grid_dep_launch();
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
    for (int t = 0; t < kRowPf; ++t) {
        if (t < per) {
            const Rec<T> v = load_rec(U, jj[t]);
            a0 += w0[t] * v.u;
            a1 += w1[t] * v.w;
            a2 += w2[t] * v.t;
            a3 += w3[t] * v.p;
        }
    }
#pragma unroll
    for (int o = kRowLanes / 2; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o, kRowLanes);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o, kRowLanes);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o, kRowLanes);
        a3 += __shfl_xor_sync(0xffffffffu, a3, o, kRowLanes);
    }
    if (!live || ln >= 4) return;
    T acc = ln == 0 ? a0 : ln == 1 ? a1 : ln == 2 ? a2 : a3;
    T b = 0;
    if (ln == 3 && tb[r]) {
        // pi'_z = g theta' / (c_p theta_bar (theta_bar + theta')) at the wall node
        T th = U[(int64_t)owner[r] * 4 + 2];
        b = gconst * th / (cp_tb2 + cp_tb2 / theta_bar * th);
    }
    res[ln * ng + pos[r]] = b - acc;
}

// u_G = W_G^{-1} r within each component, one warp per (class, position)
// computing every field of that boundary-operator class.  The kept entries
// of row (class, q) are bval[brow[r] .. brow[r+1]) at positions bcol
// (absolute, within the component), r = class * ng + q; the first
// kBandPf * 32 entries of a row are loaded before the wait.  Lanes past the
// row's end skip the product instead of multiplying a zero by some other
// component's residual: a non-finite residual (a member that has blown up
// in a batched ensemble) then stays within its own component.
constexpr int kBandPf = 4;

template <class T>
__global__ void __launch_bounds__(256) ghost_apply_band(T *__restrict__ U, int64_t ng, int64_t rows, int n_class,
                                                        const int64_t *__restrict__ brow,
                                                        const int32_t *__restrict__ bcol,
                                                        const T *__restrict__ bval, const T *__restrict__ res,
                                                        const int64_t *__restrict__ grec, int4 cls_fields) {
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const bool live = wid < (int64_t)n_class * rows;
    const int64_t w = live ? wid : 0;
    const int cls = (int)(w / rows);
    const int64_t q = w - (int64_t)cls * rows;
    const int64_t r = (int64_t)cls * ng + q;
    const int64_t b0 = __ldg(brow + r), b1 = __ldg(brow + r + 1);
    T a[kBandPf];
    int col[kBandPf];
#pragma unroll
    for (int t = 0; t < kBandPf; ++t) {
        const int64_t e = b0 + lane + 32 * t;
        const bool in = e < b1;
        a[t] = in ? __ldg(bval + e) : (T)0;
        col[t] = in ? __ldg(bcol + e) : -1;
    }
    const int fm = cls == 0 ? cls_fields.x : cls == 1 ? cls_fields.y : cls == 2 ? cls_fields.z : cls_fields.w;
    grid_dep_wait();
    grid_dep_launch();
    if (!live) return;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (!(fm & (1 << f))) continue;
        const T *rr = res + f * ng;
        T s = 0;
#pragma unroll
        for (int t = 0; t < kBandPf; ++t)
            if (col[t] >= 0) s += a[t] * rr[col[t]];
        for (int64_t e = b0 + lane + 32 * kBandPf; e < b1; e += 32) s += __ldg(bval + e) * rr[__ldg(bcol + e)];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) U[grec[q] * 4 + f] = s;
    }
}

struct UnionFind {
    std::vector<int64_t> p;
    explicit UnionFind(int64_t n) : p(n) { std::iota(p.begin(), p.end(), 0); }
    int64_t find(int64_t a) {
        while (p[a] != a) a = p[a] = p[p[a]];
        return a;
    }
    void unite(int64_t a, int64_t b) {
        a = find(a);
        b = find(b);
        if (a != b) p[std::max(a, b)] = std::min(a, b);
    }
};

}  // namespace

void build_ghost_plan(Problem &pb, const int32_t *kind_host, const int32_t *owner_host) {
    GhostPlan &gh = pb.gh;
    const int64_t ng = pb.n_all - pb.n_prog;
    gh.n_ghost = ng;
    if (ng == 0) return;
    const int n = pb.n;
    cudaStream_t st = pb.st;
    cudaEvent_t e0, e1;
    RBF_CUDA(cudaEventCreate(&e0));
    RBF_CUDA(cudaEventCreate(&e1));
    RBF_CUDA(cudaEventRecord(e0, st));

    // operator index of each BC op within pb.ops
    auto op_slot = [&](int op) {
        for (size_t i = 0; i < pb.ops.size(); ++i)
            if (pb.ops[i] == op) return (int)i;
        RBF_FAIL(RBF_E_ARG, "boundary operator %d was not built", op);
    };
    for (int64_t r = 0; r < ng; ++r) {
        int64_t b = owner_host[r];
        RBF_REQUIRE(b >= 0 && b < pb.n_prog, "ghost_owner[%lld]=%lld out of range", (long long)r, (long long)b);
        RBF_REQUIRE(kind_host[b] >= 1 && kind_host[b] <= 4, "ghost %lld is owned by a non-wall node %lld",
                    (long long)r, (long long)b);
    }
    DevBuf<int32_t> owner(ng), ridx(ng * n);
    const int nops = (int)pb.ops.size();
    DevBuf<double> rw((size_t)nops * ng * n);
    RBF_CUDA(cudaMemcpyAsync(owner.p, owner_host, ng * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    gather_rows<<<div_up(ng * n, 256), 256, 0, st>>>(pb.idx.p, pb.w64.p, nops, pb.n_prog, n, owner.p, ng, ridx.p, rw.p);
    RBF_CHECK_LAUNCH();
    std::vector<int32_t> hidx(ng * n);
    std::vector<double> hw((size_t)nops * ng * n);
    RBF_CUDA(cudaMemcpyAsync(hidx.data(), ridx.p, ridx.bytes(), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaMemcpyAsync(hw.data(), rw.p, rw.bytes(), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaStreamSynchronize(st));

    // components of the ghost coupling graph
    UnionFind uf(ng);
    std::vector<char> seen(ng, 0);
    for (int64_t r = 0; r < ng; ++r) {
        bool any = false;
        for (int k = 0; k < n; ++k) {
            int64_t j = hidx[r * n + k];
            if (j >= pb.n_prog) {
                uf.unite(r, j - pb.n_prog);
                seen[j - pb.n_prog] = 1;
                any = true;
            }
        }
        if (!any) RBF_FAIL(RBF_E_SINGULAR, "wall node %d has no ghost in its stencil", owner_host[r]);
    }
    for (int64_t g = 0; g < ng; ++g)
        if (!seen[g]) RBF_FAIL(RBF_E_SINGULAR, "ghost %lld lies in no wall node's stencil", (long long)(pb.n_prog + g));
    std::map<int64_t, int> comp_id;
    std::vector<int> comp(ng);
    for (int64_t r = 0; r < ng; ++r) {
        int64_t root = uf.find(r);
        auto it = comp_id.find(root);
        if (it == comp_id.end()) it = comp_id.emplace(root, (int)comp_id.size()).first;
        comp[r] = it->second;
    }
    const int nc = (int)comp_id.size();
    std::vector<int32_t> at(ng), pos(ng), comp_of(ng);
    std::vector<int64_t> cstart(nc + 1, 0);
    for (int64_t r = 0; r < ng; ++r) cstart[comp[r] + 1]++;
    for (int c = 0; c < nc; ++c) cstart[c + 1] += cstart[c];
    {
        std::vector<int64_t> fill(cstart.begin(), cstart.end() - 1);
        for (int64_t r = 0; r < ng; ++r) {
            int64_t q = fill[comp[r]]++;
            at[q] = (int32_t)r;
            pos[r] = (int32_t)q;
            comp_of[q] = comp[r];
        }
    }
    // boundary operator of each (row, field); fields with equal patterns share a class
    std::vector<int> wall(ng);
    for (int64_t r = 0; r < ng; ++r) {
        int kd = kind_host[owner_host[r]];
        wall[r] = (kd == 1 || kd == 2) ? 0 : 1;
    }
    std::vector<std::vector<int>> patterns;
    for (int f = 0; f < 4; ++f) {
        std::vector<int> pat(ng);
        for (int64_t r = 0; r < ng; ++r) pat[r] = kBcOps[wall[r]][f];
        int cls = -1;
        for (size_t c = 0; c < patterns.size(); ++c)
            if (patterns[c] == pat) cls = (int)c;
        if (cls < 0) {
            cls = (int)patterns.size();
            patterns.push_back(pat);
        }
        gh.field_class[f] = cls;
    }
    const int ncl = (int)patterns.size();
    gh.n_comp = nc;
    gh.n_class = ncl;
    gh.rows = ng;

    // dense W_G blocks, one per (class, component)
    std::vector<int> msize;
    std::vector<int64_t> moff;
    std::vector<double> tol;
    int64_t total = 0;
    int maxm = 0;
    for (int cl = 0; cl < ncl; ++cl)
        for (int c = 0; c < nc; ++c) {
            int m = (int)(cstart[c + 1] - cstart[c]);
            msize.push_back(m);
            moff.push_back(total);
            total += (int64_t)m * m;
            maxm = std::max(maxm, m);
        }
    RBF_REQUIRE(total < ((int64_t)1 << 31), "ghost systems too large (%lld entries)", (long long)total);
    std::vector<double> hA(total, 0.0);
    for (int cl = 0; cl < ncl; ++cl)
        for (int c = 0; c < nc; ++c) {
            int mi = cl * nc + c;
            int m = msize[mi];
            double amax = 0.0;
            for (int64_t q = cstart[c]; q < cstart[c + 1]; ++q) {
                int64_t r = at[q];
                int slot = op_slot(patterns[cl][r]);
                for (int k = 0; k < n; ++k) {
                    int64_t j = hidx[r * n + k];
                    if (j < pb.n_prog) continue;
                    int64_t col = pos[j - pb.n_prog] - cstart[c];
                    double v = hw[((size_t)slot * ng + r) * n + k];
                    hA[moff[mi] + (q - cstart[c]) * m + col] += v;
                    amax = std::max(amax, std::fabs(v));
                }
            }
            tol.push_back(1e-13 * amax);
        }
    const int nm = (int)msize.size();
    DevBuf<double> dA(total), dB(total), dcol((size_t)nm * maxm), dtol(nm);
    DevBuf<int> dms(nm), dbad(1);
    DevBuf<int64_t> dmo(nm);
    std::vector<double> hB(total, 0.0);
    for (int mi = 0; mi < nm; ++mi)
        for (int i = 0; i < msize[mi]; ++i) hB[moff[mi] + (int64_t)i * msize[mi] + i] = 1.0;
    RBF_CUDA(cudaMemcpyAsync(dA.p, hA.data(), dA.bytes(), cudaMemcpyHostToDevice, st));
    RBF_CUDA(cudaMemcpyAsync(dB.p, hB.data(), dB.bytes(), cudaMemcpyHostToDevice, st));
    RBF_CUDA(cudaMemcpyAsync(dms.p, msize.data(), nm * sizeof(int), cudaMemcpyHostToDevice, st));
    RBF_CUDA(cudaMemcpyAsync(dmo.p, moff.data(), nm * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    RBF_CUDA(cudaMemcpyAsync(dtol.p, tol.data(), nm * sizeof(double), cudaMemcpyHostToDevice, st));
    RBF_CUDA(cudaMemsetAsync(dbad.p, 0, sizeof(int), st));
    for (int k = 0; k < maxm; ++k) {
        gj_pivot<<<nm, 256, 0, st>>>(dA.p, dB.p, dms.p, dmo.p, dtol.p, k, dcol.p, maxm, dbad.p);
        dim3 grid(div_up(2 * maxm, 256) > 4 ? 4 : div_up(2 * maxm, 256), maxm, nm);
        gj_eliminate<<<grid, 256, 0, st>>>(dA.p, dB.p, dms.p, dmo.p, k, dcol.p, maxm);
    }
    RBF_CHECK_LAUNCH();
    int hbad = 0;
    RBF_CUDA(cudaMemcpyAsync(&hbad, dbad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaStreamSynchronize(st));
    if (hbad) RBF_FAIL(RBF_E_SINGULAR, "ghost system %d (class %d, component %d) is singular", hbad - 1,
                       (hbad - 1) / nc, (hbad - 1) % nc);

    const size_t ts = pb.tsize();
    gh.inv.alloc(total * ts);
    if (pb.precision == 64)
        RBF_CUDA(cudaMemcpyAsync(gh.inv.p, dB.p, dB.bytes(), cudaMemcpyDeviceToDevice, st));
    else
        to_t<float><<<div_up(total, 256), 256, 0, st>>>(dB.p, (float *)gh.inv.p, total);
    RBF_CHECK_LAUNCH();

    // per-row residual operators: BC weights with the ghost entries zeroed,
    // row-major [f][row][slot] with the slots padded to a multiple of 8
    const int npad = div_up(n, 8) * 8;
    RBF_REQUIRE(npad <= 8 * 16, "stencil too large for the ghost residual kernel");
    gh.npad = npad;
    std::vector<double> gwd((size_t)4 * npad * ng, 0.0);
    std::vector<int32_t> gidx((size_t)npad * ng);
    std::vector<unsigned char> tbv(ng);
    for (int64_t r = 0; r < ng; ++r) {
        tbv[r] = wall[r] == 0;
        for (int k = 0; k < npad; ++k) {
            int64_t j = k < n ? hidx[r * n + k] : pb.n_prog;   // padding acts like a ghost slot
            bool ghost = j >= pb.n_prog;
            gidx[(size_t)r * npad + k] = ghost ? owner_host[r] : (int32_t)j;
            for (int f = 0; f < 4; ++f) {
                int slot = op_slot(kBcOps[wall[r]][f]);
                gwd[((size_t)f * ng + r) * npad + k] = ghost ? 0.0 : hw[((size_t)slot * ng + r) * n + k];
            }
        }
    }
    gh.gidx.alloc((size_t)npad * ng);
    gh.gw.alloc((size_t)4 * npad * ng * ts);
    gh.owner.alloc(ng);
    gh.tb.alloc(ng);
    gh.pos.alloc(ng);
    gh.grec.alloc(ng);
    gh.comp_of.alloc(ng);
    gh.comp_start.alloc(nc + 1);
    gh.inv_off.alloc(nm);
    gh.res.alloc((size_t)4 * ng * ts);
    RBF_CUDA(cudaMemcpyAsync(gh.gidx.p, gidx.data(), gh.gidx.bytes(), cudaMemcpyHostToDevice, st));
    if (pb.precision == 64) {
        RBF_CUDA(cudaMemcpyAsync(gh.gw.p, gwd.data(), gwd.size() * 8, cudaMemcpyHostToDevice, st));
    } else {
        std::vector<float> gwf(gwd.begin(), gwd.end());
        RBF_CUDA(cudaMemcpyAsync(gh.gw.p, gwf.data(), gwf.size() * 4, cudaMemcpyHostToDevice, st));
        RBF_CUDA(cudaStreamSynchronize(st));
    }
    RBF_CUDA(cudaMemcpyAsync(gh.owner.p, owner_host, ng * 4, cudaMemcpyHostToDevice, st));
    RBF_CUDA(cudaMemcpyAsync(gh.tb.p, tbv.data(), ng, cudaMemcpyHostToDevice, st));
    RBF_CUDA(cudaMemcpyAsync(gh.pos.p, pos.data(), ng * 4, cudaMemcpyHostToDevice, st));
    std::vector<int64_t> grec(ng);
    for (int64_t q = 0; q < ng; ++q) grec[q] = pb.n_prog + at[q];
    RBF_CUDA(cudaMemcpyAsync(gh.grec.p, grec.data(), ng * 8, cudaMemcpyHostToDevice, st));
    RBF_CUDA(cudaStreamSynchronize(st));
    RBF_CUDA(cudaMemcpyAsync(gh.comp_of.p, comp_of.data(), ng * 4, cudaMemcpyHostToDevice, st));
    RBF_CUDA(cudaMemcpyAsync(gh.comp_start.p, cstart.data(), (nc + 1) * 8, cudaMemcpyHostToDevice, st));
    RBF_CUDA(cudaMemcpyAsync(gh.inv_off.p, moff.data(), nm * 8, cudaMemcpyHostToDevice, st));
    build_ghost_bands(gh, pb.precision, st);
    RBF_CUDA(cudaEventRecord(e1, st));
    RBF_CUDA(cudaStreamSynchronize(st));
    RBF_CUDA(cudaEventElapsedTime(&pb.ghost_setup_ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

void build_ghost_bands(GhostPlan &gh, int precision, cudaStream_t st) {
    const int64_t ng = gh.n_ghost;
    if (ng == 0) return;
    const size_t ts = precision == 64 ? 8 : 4;
    std::vector<int32_t> comp_of(ng);
    std::vector<int64_t> cstart(gh.n_comp + 1), ioff((size_t)gh.n_class * gh.n_comp);
    std::vector<unsigned char> inv(gh.inv.bytes());
    RBF_CUDA(cudaMemcpyAsync(comp_of.data(), gh.comp_of.p, ng * 4, cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaMemcpyAsync(cstart.data(), gh.comp_start.p, cstart.size() * 8, cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaMemcpyAsync(ioff.data(), gh.inv_off.p, ioff.size() * 8, cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaMemcpyAsync(inv.data(), gh.inv.p, inv.size(), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaStreamSynchronize(st));
    auto inv_at = [&](int64_t e) {
        if (precision == 64) {
            double v;
            memcpy(&v, inv.data() + e * 8, 8);
            return v;
        }
        float v;
        memcpy(&v, inv.data() + e * 4, 4);
        return (double)v;
    };
    const double thr = std::ldexp(precision == 64 ? 2.220446049250313e-16 : 1.1920928955078125e-07, -8);
    std::vector<int64_t> brow((size_t)gh.n_class * ng + 1, 0);
    std::vector<int32_t> bcol;
    std::vector<double> bval;
    for (int cl = 0; cl < gh.n_class; ++cl)
        for (int64_t q = 0; q < ng; ++q) {
            const int c = comp_of[q];
            const int64_t s0 = cstart[c];
            const int64_t m = cstart[c + 1] - s0;
            const int64_t row0 = ioff[(size_t)cl * gh.n_comp + c] + (q - s0) * m;
            double mx = 0.0;
            for (int64_t j = 0; j < m; ++j) mx = std::max(mx, std::fabs(inv_at(row0 + j)));
            for (int64_t j = 0; j < m; ++j) {
                const double v = inv_at(row0 + j);
                if (v != 0.0 && std::fabs(v) >= thr * mx) {
                    bcol.push_back((int32_t)(s0 + j));
                    bval.push_back(v);
                }
            }
            brow[(size_t)cl * ng + q + 1] = (int64_t)bcol.size();
        }
    gh.band_nnz = (int64_t)bcol.size();
    gh.brow.alloc(brow.size());
    gh.bcol.alloc(std::max<size_t>(bcol.size(), 1));
    gh.bval.alloc(std::max<size_t>(bval.size(), 1) * ts);
    RBF_CUDA(cudaMemcpyAsync(gh.brow.p, brow.data(), brow.size() * 8, cudaMemcpyHostToDevice, st));
    RBF_CUDA(cudaMemcpyAsync(gh.bcol.p, bcol.data(), bcol.size() * 4, cudaMemcpyHostToDevice, st));
    if (precision == 64) {
        RBF_CUDA(cudaMemcpyAsync(gh.bval.p, bval.data(), bval.size() * 8, cudaMemcpyHostToDevice, st));
        RBF_CUDA(cudaStreamSynchronize(st));
    } else {
        std::vector<float> bf(bval.begin(), bval.end());
        RBF_CUDA(cudaMemcpyAsync(gh.bval.p, bf.data(), bf.size() * 4, cudaMemcpyHostToDevice, st));
        RBF_CUDA(cudaStreamSynchronize(st));
    }
}

// The wall set: every prognostic node of a wall row's stencil (the records
// the ghost residual reads, the wall node itself included) and every node
// whose own stencil reads a ghost.  Only these need the stage's ghost fill
// before, or feed the next stage's ghost fill after, their stage launch.
void build_wall_set(Problem &pb) {
    const int64_t np = pb.n_prog, ng = pb.gh.n_ghost;
    const int n = pb.n;
    if (ng == 0 || pb.kind != kNS) return;
    std::vector<int32_t> idx((size_t)np * n), owner(ng);
    std::vector<unsigned char> fl(np);
    RBF_CUDA(cudaMemcpyAsync(idx.data(), pb.idx.p, idx.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, pb.st));
    RBF_CUDA(cudaMemcpyAsync(owner.data(), pb.gh.owner.p, ng * sizeof(int32_t), cudaMemcpyDeviceToHost, pb.st));
    RBF_CUDA(cudaMemcpyAsync(fl.data(), pb.flags.p, np, cudaMemcpyDeviceToHost, pb.st));
    RBF_CUDA(cudaStreamSynchronize(pb.st));
    std::vector<char> wall(np, 0);
    for (int64_t r = 0; r < ng; ++r) {
        const int64_t b = owner[r];
        wall[b] = 1;
        for (int k = 0; k < n; ++k) {
            const int64_t j = idx[b * n + k];
            if (j < np) wall[j] = 1;
        }
    }
    for (int64_t i = 0; i < np; ++i)
        for (int k = 0; k < n && !wall[i]; ++k)
            if (idx[i * n + k] >= np) wall[i] = 1;
    std::vector<int32_t> list, rest;
    for (int64_t i = 0; i < np; ++i) {
        if (wall[i]) {
            list.push_back((int32_t)i);
            fl[i] |= kWallSetFlag;
        } else {
            rest.push_back((int32_t)i);
            fl[i] &= (unsigned char)~kWallSetFlag;
        }
    }
    pb.n_wall = (int64_t)list.size();
    if (pb.n_wall == 0 || pb.n_wall == np) return;   // nothing to split
    pb.wlist.alloc(list.size());
    pb.rlist.alloc(rest.size());
    RBF_CUDA(cudaMemcpyAsync(pb.wlist.p, list.data(), list.size() * sizeof(int32_t), cudaMemcpyHostToDevice, pb.st));
    RBF_CUDA(cudaMemcpyAsync(pb.rlist.p, rest.data(), rest.size() * sizeof(int32_t), cudaMemcpyHostToDevice, pb.st));
    RBF_CUDA(cudaMemcpyAsync(pb.flags.p, fl.data(), np, cudaMemcpyHostToDevice, pb.st));
    RBF_CUDA(cudaStreamSynchronize(pb.st));
    if (!pb.side) RBF_CUDA(cudaStreamCreateWithFlags(&pb.side, cudaStreamNonBlocking));
    for (cudaEvent_t *e : {&pb.ev_fork, &pb.ev_w[0], &pb.ev_w[1], &pb.ev_r[0], &pb.ev_r[1]})
        if (!*e) RBF_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    int least = 0, greatest = 0;
    RBF_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    pb.prio_hi = greatest;
    pb.split = false;   // the autotuner, or rbf_set_stage_split, turns it on
}

void enqueue_ghost_fill(Problem &pb, void *U, cudaStream_t s, int prio) {
    GhostPlan &gh = pb.gh;
    const int64_t ng = gh.n_ghost, rows = gh.rows;
    if (ng == 0 || rows == 0) return;
    int fields[4] = {0, 0, 0, 0};
    for (int f = 0; f < 4; ++f) fields[gh.field_class[f]] |= 1 << f;
    const int4 cf = make_int4(fields[0], fields[1], fields[2], fields[3]);
    const dim3 g1(div_up(rows * kRowLanes, 256)), g2(div_up((int64_t)gh.n_class * rows * 32, 256)), blk(256);
    if (pb.precision == 64) {
        launch_kernel_prio(ghost_residual<double>, g1, blk, s, pb.pdl, prio, (const double *)U, ng, rows, gh.npad,
                      (const int32_t *)gh.gidx.p, (const double *)gh.gw.p, (const int32_t *)gh.owner.p,
                      (const unsigned char *)gh.tb.p, (const int32_t *)gh.pos.p, (double *)gh.res.p,
                      pb.cp * pb.theta_bar * pb.theta_bar, pb.theta_bar, pb.g);
        launch_kernel_prio(ghost_apply_band<double>, g2, blk, s, pb.pdl, prio, (double *)U, ng, rows, gh.n_class,
                      (const int64_t *)gh.brow.p, (const int32_t *)gh.bcol.p, (const double *)gh.bval.p,
                      (const double *)gh.res.p, (const int64_t *)gh.grec.p, cf);
    } else {
        launch_kernel_prio(ghost_residual<float>, g1, blk, s, pb.pdl, prio, (const float *)U, ng, rows, gh.npad,
                      (const int32_t *)gh.gidx.p, (const float *)gh.gw.p, (const int32_t *)gh.owner.p,
                      (const unsigned char *)gh.tb.p, (const int32_t *)gh.pos.p, (float *)gh.res.p,
                      (float)(pb.cp * pb.theta_bar * pb.theta_bar), (float)pb.theta_bar, (float)pb.g);
        launch_kernel_prio(ghost_apply_band<float>, g2, blk, s, pb.pdl, prio, (float *)U, ng, rows, gh.n_class,
                      (const int64_t *)gh.brow.p, (const int32_t *)gh.bcol.p, (const float *)gh.bval.p,
                      (const float *)gh.res.p, (const int64_t *)gh.grec.p, cf);
    }
}

}  // namespace rbf
