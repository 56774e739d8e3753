// C ABI of the GB300 library (declared in include/sbot.h): contexts, the
// slot pool, the recursive sub-cycled schedule of Algorithm 1, re-tagging,
// and state input/output.  Host code plans and launches; every step of the
// method runs in the kernels of kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/sbot.h"
#include "sbot_internal.h"
#include "topology.h"

namespace {

struct HostBody {
    int kind = 0;
    double a = 0, b = 0;
    int n = 0;
    std::vector<double> qx, qy;
    double ds = 0;
    double pivot[2] = {0, 0};
    int motion = 0;
    double x0[2] = {0, 0}, alpha_mean = 0, alpha_amp = 0, period = 1, phase = 0, heave_amp = 0, beta = 0;
    double u_ref = 1, l_ref = 1;
    int patch_side = 0;
};

struct ListRef {
    int off = 0, n = 0;
};

}  // namespace

struct sbot_ctx {
    cudaStream_t s = nullptr;
    std::string err;
    // description
    sbot_domain_desc d{};
    std::vector<RefBox> static_boxes;
    int storage = 1, B = 16, words = 8, m = 1, K = 5;
    double tau[SBOT_MAXLEV] = {};
    bool has_body = false;
    HostBody body;
    // topology
    TopoSpec ts;
    BlockStates bs;
    std::vector<PlannedBlock> planned;
    std::vector<std::vector<int>> latmap;  // per level, slot of each block position or -1
    // slot pool
    int cap = 0;
    std::vector<int> h_type, h_level, h_ox, h_oy, h_flags, h_parent, h_nbr, h_inst;
    std::vector<uint32_t> h_mask;
    std::vector<int> free_slots;
    void* f[2] = {nullptr, nullptr};
    int *d_nbr = nullptr, *d_inst = nullptr, *d_level = nullptr, *d_type = nullptr, *d_ox = nullptr, *d_oy = nullptr,
        *d_flags = nullptr, *d_parent = nullptr;
    unsigned* d_mask = nullptr;
    InstParams ip{};
    InstParams* d_ip = nullptr;
    InstState* d_ist = nullptr;
    int* d_latmap = nullptr;
    long long latmap_n = 0;
    double *d_qx = nullptr, *d_qy = nullptr;
    void* d_patch = nullptr;
    double* d_hist = nullptr;
    int* d_err = nullptr;
    int* d_lists = nullptr;
    int lists_cap = 0;
    ListRef l_fused[SBOT_MAXLEV], l_int[SBOT_MAXLEV], l_gf[SBOT_MAXLEV], l_gc[SBOT_MAXLEV];
    // split of each level's fused work: `indep` blocks read no coarse-side
    // mailbox (and, on the finest level, lie outside a static body's force
    // patch), so they run on a side stream from the start of the level's
    // sub-step, concurrently with the finer levels and the IBM; `dep` waits
    ListRef l_indep[SBOT_MAXLEV], l_dep[SBOT_MAXLEV];
    cudaStream_t side[SBOT_MAXLEV] = {};
    cudaEvent_t ev_fork[SBOT_MAXLEV] = {}, ev_join[SBOT_MAXLEV] = {};
    double bytes_indep[SBOT_MAXLEV] = {}, bytes_dep[SBOT_MAXLEV] = {};
    int* d_ibm_list = nullptr;
    size_t ibm_smem = 0;
    double* d_partials = nullptr;
    int partials_cap = 0;
    double* d_out3 = nullptr;
    // profiling: kinds 0 fused, 1 c2f, 2 f2c, 3 ibm
    int prof_mask = 0;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Rec {
        int kind;
        cudaEvent_t a, b;
        double bytes;
    };
    std::vector<Rec> pending;
    long long prof_n[4] = {};
    double prof_ms[4] = {}, prof_bytes[4] = {};
    double bytes_fused[SBOT_MAXLEV] = {}, bytes_c2f[SBOT_MAXLEV] = {}, bytes_f2c[SBOT_MAXLEV] = {};
    double bytes_ibm = 0;
    // CUDA graphs of one coarse step, one per parity of level 0 (static refinement only)
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    long long topo_version = 0, graph_version[2] = {-1, -1};
    int graph_mask[2] = {-1, -1};
    std::vector<Rec> graph_recs[2];  // profiling events recorded inside the graph
    bool capturing = false;
    bool own_stream = false;
    int device = 0;
    // time
    int par[SBOT_MAXLEV] = {};
    bool finalized = false;
    long long coarse_step = 0;
    long long forces_read = 0;
};

namespace {

sbot_status fail(sbot_ctx* c, sbot_status st, const std::string& m) {
    if (c) c->err = m;
    return st;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(c, SBOT_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMalloc((void**)p, n * sizeof(T));
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

DevPool pool_view(sbot_ctx* c) {
    DevPool P;
    P.B = c->B;
    P.mask_words = c->words;
    P.nbr = c->d_nbr;
    P.slot_inst = c->d_inst;
    P.slot_level = c->d_level;
    P.slot_type = c->d_type;
    P.slot_ox = c->d_ox;
    P.slot_oy = c->d_oy;
    P.slot_flags = c->d_flags;
    P.slot_parent = c->d_parent;
    P.slot_mask = c->d_mask;
    P.inst = c->d_ip;
    P.ist = c->d_ist;
    P.latmap = c->d_latmap;
    P.mk_qx = c->d_qx;
    P.mk_qy = c->d_qy;
    P.patch = c->d_patch;
    P.hist = c->d_hist;
    P.err = c->d_err;
    return P;
}

// Sec. 3.6 kinematics, for planning on the host (the kernels evaluate it again)
void host_pose(const HostBody& b, double t, double& cx, double& cy, double& al) {
    al = b.alpha_mean;
    double hx = 0, hy = 0;
    if (b.motion >= 1) al = b.alpha_mean - b.alpha_amp * std::sin(2.0 * M_PI * t / b.period + b.phase);
    if (b.motion == 2) {
        double h = 0.5 * b.heave_amp * std::cos(2.0 * M_PI * t / b.period);
        hx = h * std::cos(b.beta);
        hy = h * std::sin(b.beta);
    }
    cx = b.x0[0] + hx;
    cy = b.x0[1] + hy;
}

// markers at equal arc length: the perimeter is the length of the polygon of
// 64 n vertices at equal parameter steps t_k = 2 pi k / (64 n) on
// (a cos t, b sin t); marker j sits at arc length j P / n, its parameter
// interpolated linearly inside the polygon edge that holds it.  A circle is
// placed at equal angles directly.
double place_markers(double a, double b, int n, std::vector<double>& qx, std::vector<double>& qy) {
    qx.resize(n);
    qy.resize(n);
    if (a == b) {
        for (int j = 0; j < n; j++) {
            double t = 2.0 * M_PI * j / n;
            qx[j] = a * std::cos(t);
            qy[j] = a * std::sin(t);
        }
        return 2.0 * M_PI * a;
    }
    const int M = 64 * n;
    std::vector<double> arc(M + 1, 0.0);
    for (int k = 0; k < M; k++) {
        double t0 = 2.0 * M_PI * k / M, t1 = 2.0 * M_PI * (k + 1) / M;
        double ex = a * std::cos(t1) - a * std::cos(t0), ey = b * std::sin(t1) - b * std::sin(t0);
        arc[k + 1] = arc[k] + std::sqrt(ex * ex + ey * ey);
    }
    double P = arc[M];
    int k = 0;
    for (int j = 0; j < n; j++) {
        double want = P * j / n;
        while (k < M - 1 && arc[k + 1] <= want) k++;
        double fr = (want - arc[k]) / (arc[k + 1] - arc[k]);
        double t = 2.0 * M_PI * (k + fr) / M;
        qx[j] = a * std::cos(t);
        qy[j] = b * std::sin(t);
    }
    return P;
}

// refinement boxes of the coarse step [n, n+1]: static ones plus the body's
// marker bounding box over its finest steps, widened per level
void window_boxes(sbot_ctx* c, long long n, std::vector<RefBox>& out) {
    out = c->static_boxes;
    if (!c->has_body) return;
    const HostBody& b = c->body;
    long long nf = 1LL << (c->m - 1);
    double mnx = 1e300, mny = 1e300, mxx = -1e300, mxy = -1e300;
    for (long long k = n * nf; k <= (n + 1) * nf; k++) {
        double cx, cy, al;
        host_pose(b, (double)k, cx, cy, al);
        double ca = std::cos(al), sa = std::sin(al);
        for (int j = 0; j < b.n; j++) {
            double px = b.qx[j] - b.pivot[0], py = b.qy[j] - b.pivot[1];
            double rx = cx + b.pivot[0] + ca * px - sa * py;
            double ry = cy + b.pivot[1] + sa * px + ca * py;
            mnx = std::min(mnx, rx);
            mxx = std::max(mxx, rx);
            mny = std::min(mny, ry);
            mxy = std::max(mxy, ry);
        }
    }
    for (int l = 1; l < c->m; l++) {
        double g = c->d.refine_margin[l];
        if (g <= 0) continue;
        out.push_back({l, mnx - g, mny - g, mxx + g + c->d.refine_wake[l], mxy + g});
    }
}

sbot_status grow_pool(sbot_ctx* c, int need) {
    if (need <= c->cap) return SBOT_OK;
    int ncap = std::max(need, c->cap + c->cap / 2);
    size_t per = (size_t)9 * c->B * c->B * storage_bytes(c->storage);
    void* nf[2] = {nullptr, nullptr};
    for (int i = 0; i < 2; i++) {
        if (cudaMalloc(&nf[i], (size_t)ncap * per) != cudaSuccess) {
            cudaGetLastError();
            dfree(nf[0]);
            return fail(c, SBOT_ERR_OOM, "population pool allocation failed");
        }
        if (c->f[i]) {
            CK(cudaMemcpyAsync(nf[i], c->f[i], (size_t)c->cap * per, cudaMemcpyDeviceToDevice, c->s));
        }
    }
    CK(cudaStreamSynchronize(c->s));
    for (int i = 0; i < 2; i++) {
        dfree(c->f[i]);
        c->f[i] = nf[i];
    }
    for (int sl = ncap - 1; sl >= c->cap; sl--) c->free_slots.push_back(sl);
    c->h_type.resize(ncap, ST_FREE);
    c->h_level.resize(ncap, 0);
    c->h_ox.resize(ncap, 0);
    c->h_oy.resize(ncap, 0);
    c->h_flags.resize(ncap, 0);
    c->h_parent.resize(ncap, -1);
    c->h_inst.resize(ncap, 0);
    c->h_nbr.resize((size_t)ncap * 9, -1);
    c->h_mask.resize((size_t)ncap * c->words, 0u);
    dfree(c->d_nbr);
    dfree(c->d_inst);
    dfree(c->d_level);
    dfree(c->d_type);
    dfree(c->d_ox);
    dfree(c->d_oy);
    dfree(c->d_flags);
    dfree(c->d_parent);
    dfree(c->d_mask);
    CK(dalloc(&c->d_nbr, (size_t)ncap * 9));
    CK(dalloc(&c->d_inst, ncap));
    CK(dalloc(&c->d_level, ncap));
    CK(dalloc(&c->d_type, ncap));
    CK(dalloc(&c->d_ox, ncap));
    CK(dalloc(&c->d_oy, ncap));
    CK(dalloc(&c->d_flags, ncap));
    CK(dalloc(&c->d_parent, ncap));
    CK(dalloc(&c->d_mask, (size_t)ncap * c->words));
    c->cap = ncap;
    return SBOT_OK;
}

int popcount_mask(const std::vector<uint32_t>& m);

struct RetagJob {
    int v[8];  // dst, kind, sources x4, source buffer, destination buffer
};

// Build (or rebuild) the topology for the coarse step [n, n+1].  With
// `transfer`, interior blocks that stay keep their slot and state, and new
// interior blocks get the post-collision state of the old grid (reading R5):
// a copy of the covering coarser cell, or the mean of the 4 children.
sbot_status build_topology(sbot_ctx* c, long long n, bool transfer, bool* changed) {
    if (changed) *changed = false;
    TopoSpec ts;
    ts.m = c->m;
    ts.B = c->B;
    ts.nx0 = c->d.nx0;
    ts.ny0 = c->d.ny0;
    ts.periodic_x = c->d.bc[SIDE_W] == BCK_PERIODIC;
    ts.periodic_y = c->d.bc[SIDE_S] == BCK_PERIODIC;
    window_boxes(c, n, ts.boxes);
    BlockStates bs;
    const char* why = nullptr;
    if (!plan_blocks(ts, bs, &why)) return fail(c, SBOT_ERR_STATE, why);
    if (transfer && !c->bs.s.empty() && bs.s == c->bs.s) return SBOT_OK;
    if (changed) *changed = true;
    std::vector<PlannedBlock> planned;
    plan_slots(ts, bs, planned);

    const BlockStates old = c->bs;
    const std::vector<std::vector<int>> old_lat = c->latmap;
    const bool have_old = transfer && !old.s.empty();

    // slots: interior blocks that remain interior keep theirs
    std::vector<int> keep_slot(planned.size(), -1);
    std::vector<char> still_used(c->cap, 0);
    if (have_old) {
        for (size_t i = 0; i < planned.size(); i++) {
            const PlannedBlock& pb = planned[i];
            if (pb.type != ST_INT || old.at(pb.level, pb.bx, pb.by) != 1) continue;
            int sl = old_lat[pb.level][(size_t)pb.by * old.nbx[pb.level] + pb.bx];
            keep_slot[i] = sl;
            still_used[sl] = 1;
        }
    }
    // old slots that are not kept: halo / mailbox slots are free now; old
    // interior slots are freed after the transfer has read them
    std::vector<int> release_after;
    for (int sl = 0; sl < c->cap; sl++) {
        if (c->h_type[sl] == ST_FREE || still_used[sl]) continue;
        if (c->h_type[sl] == ST_INT && have_old)
            release_after.push_back(sl);
        else {
            c->h_type[sl] = ST_FREE;
            c->free_slots.push_back(sl);
        }
    }
    int need_new = 0;
    for (size_t i = 0; i < planned.size(); i++)
        if (keep_slot[i] < 0) need_new++;
    int in_use = c->cap - (int)c->free_slots.size();
    if ((int)c->free_slots.size() < need_new) {
        sbot_status st = grow_pool(c, in_use + need_new + 16);
        if (st != SBOT_OK) return st;
    }
    std::sort(c->free_slots.begin(), c->free_slots.end(), std::greater<int>());
    std::vector<int> slot_of(planned.size());
    for (size_t i = 0; i < planned.size(); i++) {
        if (keep_slot[i] >= 0) {
            slot_of[i] = keep_slot[i];
        } else {
            slot_of[i] = c->free_slots.back();
            c->free_slots.pop_back();
        }
    }
    // lattice maps
    std::vector<std::vector<int>> lat(c->m);
    for (int l = 0; l < c->m; l++) lat[l].assign((size_t)bs.nbx[l] * bs.nby[l], -1);
    for (size_t i = 0; i < planned.size(); i++)
        lat[planned[i].level][(size_t)planned[i].by * bs.nbx[planned[i].level] + planned[i].bx] = slot_of[i];
    // transfer jobs for new interior blocks
    std::vector<RetagJob> jobs;
    if (have_old) {
        for (size_t i = 0; i < planned.size(); i++) {
            const PlannedBlock& pb = planned[i];
            if (pb.type != ST_INT || keep_slot[i] >= 0) continue;
            int l = pb.level, ost = old.at(l, pb.bx, pb.by);
            RetagJob j{};
            j.v[0] = slot_of[i];
            if (ost == 0) {  // was inside a coarser leaf
                int ll = l, bx = pb.bx, by = pb.by;
                while (ll > 0) {
                    ll--;
                    bx >>= 1;
                    by >>= 1;
                    if (old.at(ll, bx, by) == 1) break;
                }
                if (old.at(ll, bx, by) != 1) return fail(c, SBOT_ERR_STATE, "re-tag: no covering coarser block");
                j.v[1] = 0;
                j.v[2] = old_lat[ll][(size_t)by * old.nbx[ll] + bx];
                j.v[3] = l - ll;
                j.v[6] = c->par[ll];
            } else {  // was refined: mean of the children (one level down)
                j.v[1] = 1;
                for (int qd = 0; qd < 4; qd++) {
                    int cbx = 2 * pb.bx + (qd & 1), cby = 2 * pb.by + (qd >> 1);
                    if (l + 1 >= c->m || old.at(l + 1, cbx, cby) != 1)
                        return fail(c, SBOT_ERR_STATE, "re-tag changed a region by more than one level in one step");
                    j.v[2 + qd] = old_lat[l + 1][(size_t)cby * old.nbx[l + 1] + cbx];
                }
                j.v[6] = c->par[l + 1];
            }
            j.v[7] = c->par[l];
            jobs.push_back(j);
        }
    }
    // slot tables
    for (size_t i = 0; i < planned.size(); i++) {
        const PlannedBlock& pb = planned[i];
        int sl = slot_of[i];
        c->h_type[sl] = pb.type;
        c->h_level[sl] = pb.level;
        c->h_inst[sl] = 0;
        c->h_ox[sl] = pb.bx * c->B;
        c->h_oy[sl] = pb.by * c->B;
        int l = pb.level;
        bool edge = (!ts.periodic_x && (pb.bx == 0 || pb.bx == bs.nbx[l] - 1)) ||
                    (!ts.periodic_y && (pb.by == 0 || pb.by == bs.nby[l] - 1));
        c->h_flags[sl] = edge ? SLOTF_EDGE : 0;
        c->h_parent[sl] = (pb.type == ST_GF) ? lat[l - 1][(size_t)(pb.by >> 1) * bs.nbx[l - 1] + (pb.bx >> 1)] : -1;
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int x = pb.bx + dx, y = pb.by + dy, v = -1;
                bool inx = x >= 0 && x < bs.nbx[l], iny = y >= 0 && y < bs.nby[l];
                if (!inx && ts.periodic_x) {
                    x = (x + bs.nbx[l]) % bs.nbx[l];
                    inx = true;
                }
                if (!iny && ts.periodic_y) {
                    y = (y + bs.nby[l]) % bs.nby[l];
                    iny = true;
                }
                if (inx && iny) v = lat[l][(size_t)y * bs.nbx[l] + x];
                c->h_nbr[(size_t)sl * 9 + (dy + 1) * 3 + (dx + 1)] = v;
            }
        std::copy(pb.mask.begin(), pb.mask.end(), c->h_mask.begin() + (size_t)sl * c->words);
    }
    // upload tables (the old interior slots that feed the transfer keep their entries)
    cudaStream_t s = c->s;
    CK(cudaMemcpyAsync(c->d_nbr, c->h_nbr.data(), c->h_nbr.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_inst, c->h_inst.data(), c->cap * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_level, c->h_level.data(), c->cap * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_type, c->h_type.data(), c->cap * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_ox, c->h_ox.data(), c->cap * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_oy, c->h_oy.data(), c->cap * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_flags, c->h_flags.data(), c->cap * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_parent, c->h_parent.data(), c->cap * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_mask, c->h_mask.data(), c->h_mask.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    // lattice map
    long long tot = 0;
    for (int l = 0; l < c->m; l++) {
        c->ip.latmap_off[l] = tot;
        c->ip.nbx[l] = bs.nbx[l];
        c->ip.nby[l] = bs.nby[l];
        tot += (long long)lat[l].size();
    }
    if (tot > c->latmap_n) {
        dfree(c->d_latmap);
        CK(dalloc(&c->d_latmap, (size_t)tot));
        c->latmap_n = tot;
    }
    std::vector<int> flat;
    flat.reserve(tot);
    for (int l = 0; l < c->m; l++) flat.insert(flat.end(), lat[l].begin(), lat[l].end());
    CK(cudaMemcpyAsync(c->d_latmap, flat.data(), tot * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_ip, &c->ip, sizeof(InstParams), cudaMemcpyHostToDevice, s));
    // which interior blocks must wait: a mailbox neighbour (coarse side of an
    // interface), or, on the finest level, the force patch of a static body
    std::vector<char> dep(planned.size(), 0);
    int bx0 = 1 << 30, by0 = 1 << 30, bx1 = -1, by1 = -1;  // static body stencil box, finest cells
    bool static_body = c->has_body && c->body.motion == 0;
    if (static_body) {
        double cs = std::cos(c->body.alpha_mean), sn = std::sin(c->body.alpha_mean);
        for (int j = 0; j < c->body.n; j++) {
            double px = c->body.qx[j] - c->body.pivot[0], py = c->body.qy[j] - c->body.pivot[1];
            double rx = c->body.x0[0] + c->body.pivot[0] + cs * px - sn * py;
            double ry = c->body.x0[1] + c->body.pivot[1] + sn * px + cs * py;
            int i0 = (int)std::floor(rx - 0.5) - 1, j0 = (int)std::floor(ry - 0.5) - 1;
            bx0 = std::min(bx0, i0 - 1);
            by0 = std::min(by0, j0 - 1);
            bx1 = std::max(bx1, i0 + 4);
            by1 = std::max(by1, j0 + 4);
        }
    }
    for (size_t i = 0; i < planned.size(); i++) {
        const PlannedBlock& pb = planned[i];
        if (pb.type != ST_INT) continue;
        int sl = slot_of[i];
        for (int k = 0; k < 9; k++) {
            int nb = c->h_nbr[(size_t)sl * 9 + k];
            if (nb >= 0 && c->h_type[nb] == ST_GC) dep[i] = 1;
        }
        if (pb.level == c->m - 1 && c->has_body) {
            if (!static_body) {
                dep[i] = 1;
            } else {
                int x0 = pb.bx * c->B, y0 = pb.by * c->B;
                if (x0 <= bx1 && bx0 < x0 + c->B && y0 <= by1 && by0 < y0 + c->B) dep[i] = 1;
            }
        }
    }
    // work lists per level
    std::vector<int> lists;
    for (int l = 0; l < c->m; l++) {
        auto add = [&](ListRef& r, auto pred) {
            r.off = (int)lists.size();
            for (size_t i = 0; i < planned.size(); i++)
                if (planned[i].level == l && pred(planned[i].type, dep[i])) lists.push_back(slot_of[i]);
            r.n = (int)lists.size() - r.off;
        };
        add(c->l_int[l], [](int t, char) { return t == ST_INT; });
        add(c->l_fused[l], [](int t, char) { return t == ST_INT || t == ST_GF; });
        add(c->l_gf[l], [](int t, char) { return t == ST_GF; });
        add(c->l_gc[l], [](int t, char) { return t == ST_GC; });
        add(c->l_indep[l], [](int t, char d) { return (t == ST_INT && !d) || t == ST_GF; });
        add(c->l_dep[l], [](int t, char d) { return t == ST_INT && d; });
    }
    size_t jobs_ints = jobs.size() * 8;
    if ((int)(lists.size() + jobs_ints) > c->lists_cap) {
        dfree(c->d_lists);
        c->lists_cap = (int)(lists.size() + jobs_ints) * 2 + 64;
        CK(dalloc(&c->d_lists, c->lists_cap));
    }
    CK(cudaMemcpyAsync(c->d_lists, lists.data(), lists.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    if (!jobs.empty()) {
        int* d_jobs = c->d_lists + lists.size();
        CK(cudaMemcpyAsync(d_jobs, jobs.data(), jobs_ints * sizeof(int), cudaMemcpyHostToDevice, s));
        DevPool P = pool_view(c);
        // at the start of a coarse step every level holds its post-collision state in f[par[l]]
        launch_retag(c->storage, P, d_jobs, (int)jobs.size(), c->f[0], c->f[1], s);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));
    }
    for (int sl : release_after) {
        c->h_type[sl] = ST_FREE;
        c->free_slots.push_back(sl);
    }
    if (!release_after.empty())
        CK(cudaMemcpyAsync(c->d_type, c->h_type.data(), c->cap * sizeof(int), cudaMemcpyHostToDevice, s));
    c->ts = ts;
    c->bs = bs;
    c->planned = planned;
    c->latmap = lat;
    // algorithmic bytes per launch: every interior or halo cell reads and
    // writes its 9 populations once; the merge reads 4 fine and writes 1
    // coarse value per mailbox population; the IBM pulls its patch once
    double sb = storage_bytes(c->storage);
    for (int l = 0; l < c->m; l++) {
        double cells_int = 0, cells_gf = 0, cells_gc = 0;
        for (const PlannedBlock& pb : planned) {
            if (pb.level != l) continue;
            if (pb.type == ST_INT) cells_int += (double)c->B * c->B;
            if (pb.type == ST_GF) cells_gf += popcount_mask(pb.mask);
            if (pb.type == ST_GC) cells_gc += popcount_mask(pb.mask);
        }
        c->bytes_fused[l] = (cells_int + cells_gf) * 18.0 * sb;
        c->bytes_dep[l] = (double)c->l_dep[l].n * c->B * c->B * 18.0 * sb;
        c->bytes_indep[l] = c->bytes_fused[l] - c->bytes_dep[l];
        c->bytes_c2f[l] = cells_gf * 18.0 * sb;
        c->bytes_f2c[l] = cells_gc * 3.0 * 5.0 * sb;  // ~3 populations per mailbox cell, 4 reads + 1 write
    }
    c->bytes_ibm = c->has_body ? (double)c->ip.patch_cap * 9.0 * sb : 0.0;
    c->topo_version++;
    return SBOT_OK;
}

sbot_status finalize_init(sbot_ctx* c) {
    if (c->finalized) return SBOT_OK;
    DevPool P = pool_view(c);
    int fin = c->m - 1;
    // pre-collision state at t = 0 lives in f[1]; collide it into f[0]
    if (c->has_body) {
        launch_ibm(c->storage, P, c->d_ibm_list, 1, c->f[1], fin, 1, c->ibm_smem, c->s);
        CK(cudaGetLastError());
    }
    for (int l = 0; l < c->m; l++) {
        launch_collide_init(c->storage, P, c->d_lists + c->l_int[l].off, c->l_int[l].n, c->f[1], c->f[0], l, c->s);
        c->par[l] = 0;
    }
    CK(cudaGetLastError());
    c->finalized = true;
    return SBOT_OK;
}

cudaEvent_t next_event(sbot_ctx* c) {
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

struct ProfScope {
    sbot_ctx* c;
    int kind;
    double bytes;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    // direct launches draw events from a reusable pool; a graph being captured
    // gets its own events (external record nodes), destroyed with the graph
    cudaEvent_t ev() {
        if (!c->capturing) return next_event(c);
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    ProfScope(sbot_ctx* c_, int k, double b, cudaStream_t s_ = nullptr) : c(c_), kind(k), bytes(b), st(s_ ? s_ : c_->s) {
        if (c->prof_mask & (1 << kind)) {
            a = ev();
            cudaEventRecordWithFlags(a, st, c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
        }
    }
    ~ProfScope() {
        if (!a) return;
        cudaEvent_t b = ev();
        cudaEventRecordWithFlags(b, st, c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
        c->pending.push_back({kind, a, b, bytes});
    }
};

void resolve_profile(sbot_ctx* c) {
    if (c->pending.empty()) return;
    cudaEventSynchronize(c->pending.back().b);
    for (auto& r : c->pending) {
        float ms = 0;
        cudaEventElapsedTime(&ms, r.a, r.b);
        c->prof_n[r.kind]++;
        c->prof_ms[r.kind] += ms;
        c->prof_bytes[r.kind] += r.bytes;
    }
    c->pending.clear();
    c->ev_used = 0;
}

void drop_graph(sbot_ctx* c, int g) {
    if (c->gexec[g]) cudaGraphExecDestroy(c->gexec[g]);
    c->gexec[g] = nullptr;
    for (auto& r : c->graph_recs[g]) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    c->graph_recs[g].clear();
}

// events recorded by a graph replay: read them (after the replay finished)
void resolve_graph_profile(sbot_ctx* c, int g) {
    if (c->graph_recs[g].empty()) return;
    cudaEventSynchronize(c->graph_recs[g].back().b);
    for (auto& r : c->graph_recs[g]) {
        float ms = 0;
        cudaEventElapsedTime(&ms, r.a, r.b);
        c->prof_n[r.kind]++;
        c->prof_ms[r.kind] += ms;
        c->prof_bytes[r.kind] += r.bytes;
    }
}

// one substep of level l (and, recursively, two of every finer level):
// Algorithm 1 with each stream+collide pair fused into one pull kernel
void advance(sbot_ctx* c, const DevPool& P, int l) {
    int storage = c->storage;
    const bool fork = c->l_indep[l].n > 0 && c->l_dep[l].n > 0 && c->side[l];
    if (fork) {
        cudaEventRecord(c->ev_fork[l], c->s);
        cudaStreamWaitEvent(c->side[l], c->ev_fork[l], 0);
        {
            ProfScope ps(c, 0, c->bytes_indep[l], c->side[l]);
            launch_fused(storage, P, c->d_lists + c->l_indep[l].off, c->l_indep[l].n, c->f[c->par[l]],
                         c->f[1 - c->par[l]], l, c->side[l], 0);
        }
        cudaEventRecord(c->ev_join[l], c->side[l]);
    }
    if (l + 1 < c->m) {
        {
            ProfScope ps(c, 1, c->bytes_c2f[l + 1]);
            launch_c2f(storage, P, c->d_lists + c->l_gf[l + 1].off, c->l_gf[l + 1].n, c->f[c->par[l]],
                       c->f[c->par[l + 1]], c->s);
        }
        advance(c, P, l + 1);
        advance(c, P, l + 1);
        {
            ProfScope ps(c, 2, c->bytes_f2c[l]);
            launch_f2c(storage, P, c->d_lists + c->l_gc[l].off, c->l_gc[l].n, c->f[c->par[l]],
                       c->f[c->par[l + 1]], l, c->s);
        }
    }
    if (c->has_body && l == c->m - 1) {
        ProfScope ps(c, 3, c->bytes_ibm);
        launch_ibm(storage, P, c->d_ibm_list, 1, c->f[c->par[l]], l, 0, c->ibm_smem, c->s);
    }
    if (fork) {
        {
            ProfScope ps(c, 0, c->bytes_dep[l]);
            launch_fused(storage, P, c->d_lists + c->l_dep[l].off, c->l_dep[l].n, c->f[c->par[l]],
                         c->f[1 - c->par[l]], l, c->s, 1);
        }
        cudaStreamWaitEvent(c->s, c->ev_join[l], 0);
    } else {
        ProfScope ps(c, 0, c->bytes_fused[l]);
        launch_fused(storage, P, c->d_lists + c->l_fused[l].off, c->l_fused[l].n, c->f[c->par[l]],
                     c->f[1 - c->par[l]], l, c->s);
    }
    c->par[l] ^= 1;
}

int popcount_mask(const std::vector<uint32_t>& m) {
    int n = 0;
    for (uint32_t w : m) n += __builtin_popcount(w);
    return n;
}

sbot_status check_device_error(sbot_ctx* c) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (e == 0) return SBOT_OK;
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->s));
    std::string m = "device reported:";
    if (e & ERRB_STENCIL) m += " a marker stencil left the finest interior cells;";
    if (e & ERRB_PATCH) m += " the marker patch exceeded its capacity;";
    if (e & ERRB_NOSOURCE) m += " an interior cell found no streaming source;";
    if (e & ERRB_HALO) m += " a coalescence found no fine halo cell;";
    if (e & ERRB_NONFINITE) return fail(c, SBOT_ERR_NONFINITE, m + " non-finite populations");
    return fail(c, SBOT_ERR_STATE, m);
}

sbot_status level_ok(sbot_ctx* c, int level) {
    if (level < 0 || level >= c->m) return fail(c, SBOT_ERR_ARG, "level out of range");
    return SBOT_OK;
}

sbot_status upload_dense_pre(sbot_ctx* c, int level, const double* host, int planes, int from_fields) {
    int nx = c->d.nx0 << level, ny = c->d.ny0 << level;
    long long plane = (long long)nx * ny;
    double* d = nullptr;
    CK(dalloc(&d, (size_t)planes * plane));
    CK(cudaMemcpyAsync(d, host, (size_t)planes * plane * sizeof(double), cudaMemcpyHostToDevice, c->s));
    DevPool P = pool_view(c);
    launch_set_pre(c->storage, P, c->d_lists + c->l_int[level].off, c->l_int[level].n, c->f[1], nx, d, plane,
                   from_fields, c->s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->s));
    dfree(d);
    return SBOT_OK;
}

sbot_status reset_state(sbot_ctx* c) {
    DevPool P = pool_view(c);
    for (int l = 0; l < c->m; l++)
        launch_set_pre(c->storage, P, c->d_lists + c->l_int[l].off, c->l_int[l].n, c->f[1], 0, nullptr, 0, 1, c->s);
    CK(cudaGetLastError());
    InstState z{};
    CK(cudaMemcpyAsync(c->d_ist, &z, sizeof(InstState), cudaMemcpyHostToDevice, c->s));
    c->finalized = false;
    c->coarse_step = 0;
    c->forces_read = 0;
    for (int l = 0; l < SBOT_MAXLEV; l++) c->par[l] = 0;
    return SBOT_OK;
}

// dense export of level `level`: mode 0 populations, mode 1 fields
sbot_status export_level(sbot_ctx* c, int level, int mode, std::vector<double>& out) {
    sbot_status st = finalize_init(c);
    if (st != SBOT_OK) return st;
    int nx = c->d.nx0 << level, ny = c->d.ny0 << level;
    long long plane = (long long)nx * ny;
    int planes = mode == 0 ? 9 : 3;
    double* d = nullptr;
    CK(dalloc(&d, (size_t)planes * plane));
    CK(cudaMemsetAsync(d, 0, (size_t)planes * plane * sizeof(double), c->s));
    DevPool P = pool_view(c);
    bool direct = c->coarse_step == 0;
    const void* src = direct ? c->f[1] : c->f[1 - c->par[level]];
    launch_export(c->storage, P, c->d_lists + c->l_int[level].off, c->l_int[level].n, src, level, direct ? 1 : 0, nx,
                  d, plane, mode, c->s);
    CK(cudaGetLastError());
    out.resize((size_t)planes * plane);
    CK(cudaMemcpyAsync(out.data(), d, out.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    dfree(d);
    return check_device_error(c);
}

sbot_status validate_desc(const sbot_domain_desc* d, std::string& why) {
    if (!d) return why = "null description", SBOT_ERR_ARG;
    if (d->levels < 1 || d->levels > SBOT_MAXLEV) return why = "levels must be 1..8", SBOT_ERR_ARG;
    if (d->block != 8 && d->block != 16 && d->block != 32) return why = "block must be 8, 16 or 32", SBOT_ERR_ARG;
    if (d->nx0 <= 0 || d->ny0 <= 0 || d->nx0 % d->block || d->ny0 % d->block)
        return why = "nx0, ny0 must be positive multiples of block", SBOT_ERR_ARG;
    for (int i = 0; i < 4; i++)
        if (d->bc[i] < 0 || d->bc[i] > 3) return why = "bad boundary kind", SBOT_ERR_ARG;
    if ((d->bc[0] == 0) != (d->bc[1] == 0) || (d->bc[2] == 0) != (d->bc[3] == 0))
        return why = "opposite sides must both be periodic or both not", SBOT_ERR_ARG;
    if (!(d->tau_finest > 0.5)) return why = "tau must exceed 1/2", SBOT_ERR_ARG;
    if (d->storage < 0 || d->storage > 3) return why = "bad storage kind", SBOT_ERR_ARG;
    if (d->n_boxes < 0 || (d->n_boxes > 0 && !d->boxes)) return why = "bad refinement boxes", SBOT_ERR_ARG;
    long long cells = (long long)d->nx0 * d->ny0 << (2 * (d->levels - 1));
    if (cells > (1LL << 36)) return why = "domain too large", SBOT_ERR_ARG;
    return SBOT_OK;
}

}  // namespace

extern "C" {

sbot_status sbot_create_domain(const sbot_domain_desc* desc, void* cuda_stream, sbot_ctx_t* out) {
    std::string why;
    if (!out) return SBOT_ERR_ARG;
    *out = nullptr;
    sbot_status vs = validate_desc(desc, why);
    if (vs != SBOT_OK) return vs;
    sbot_ctx* c = new sbot_ctx();
    cudaGetDevice(&c->device);
    c->s = (cudaStream_t)cuda_stream;
    if (!c->s) {
        if (cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return SBOT_ERR_CUDA;
        }
        c->own_stream = true;
    }
    c->d = *desc;
    c->d.boxes = nullptr;
    for (int i = 0; i < desc->n_boxes; i++)
        c->static_boxes.push_back({desc->boxes[i].level, desc->boxes[i].x0, desc->boxes[i].y0, desc->boxes[i].x1,
                                   desc->boxes[i].y1});
    c->storage = desc->storage;
    c->B = desc->block;
    c->words = (c->B * c->B + 31) / 32;
    c->m = desc->levels;
    c->K = desc->ibm_iters > 0 ? desc->ibm_iters : 5;
    InstParams& ip = c->ip;
    ip.m = c->m;
    ip.nx0 = desc->nx0;
    ip.ny0 = desc->ny0;
    for (int i = 0; i < 4; i++) ip.bc[i] = desc->bc[i];
    ip.periodic_x = desc->bc[SIDE_W] == BCK_PERIODIC;
    ip.periodic_y = desc->bc[SIDE_S] == BCK_PERIODIC;
    for (int l = 0; l < c->m; l++) {
        // acoustic scaling (Eq. 9 per level): nu halves with every finer level
        ip.tau[l] = 0.5 + (desc->tau_finest - 0.5) / (double)(1 << (c->m - 1 - l));
        c->tau[l] = ip.tau[l];
    }
    ip.rho0 = desc->rho0;
    ip.uin_x = desc->u_in[0];
    ip.uin_y = desc->u_in[1];
    ip.K = c->K;
    ip.hist_off = 0;
    sbot_status st = SBOT_OK;
    auto bail = [&](sbot_status e) {
        sbot_destroy(c);
        return e;
    };
    for (int l = 0; l < c->m; l++) {
        if (cudaStreamCreateWithFlags(&c->side[l], cudaStreamNonBlocking) != cudaSuccess) return bail(SBOT_ERR_CUDA);
        if (cudaEventCreateWithFlags(&c->ev_fork[l], cudaEventDisableTiming) != cudaSuccess) return bail(SBOT_ERR_CUDA);
        if (cudaEventCreateWithFlags(&c->ev_join[l], cudaEventDisableTiming) != cudaSuccess) return bail(SBOT_ERR_CUDA);
    }
    if (cudaMalloc((void**)&c->d_ip, sizeof(InstParams)) != cudaSuccess) return bail(SBOT_ERR_OOM);
    if (cudaMalloc((void**)&c->d_ist, sizeof(InstState)) != cudaSuccess) return bail(SBOT_ERR_OOM);
    if (cudaMalloc((void**)&c->d_err, sizeof(int)) != cudaSuccess) return bail(SBOT_ERR_OOM);
    if (cudaMalloc((void**)&c->d_out3, 3 * sizeof(double)) != cudaSuccess) return bail(SBOT_ERR_OOM);
    if (cudaMalloc((void**)&c->d_ibm_list, sizeof(int)) != cudaSuccess) return bail(SBOT_ERR_OOM);
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->s);
    cudaMemsetAsync(c->d_ibm_list, 0, sizeof(int), c->s);
    st = build_topology(c, 0, false, nullptr);
    if (st != SBOT_OK) {
        why = c->err;
        sbot_destroy(c);
        return st;
    }
    st = reset_state(c);
    if (st != SBOT_OK) return bail(st);
    *out = c;
    return SBOT_OK;
}

static bool host_body_from_desc(const sbot_body_desc* b, HostBody& hb) {
    if (b->n_markers < 3 || b->a <= 0 || (b->kind == 1 && b->b <= 0) || !(b->period > 0)) return false;
    hb.kind = b->kind;
    hb.a = b->a;
    hb.b = b->kind == 0 ? b->a : b->b;
    hb.n = b->n_markers;
    double P = place_markers(hb.a, hb.b, hb.n, hb.qx, hb.qy);
    hb.ds = P / hb.n;  // Delta s_b = perimeter / n
    hb.pivot[0] = b->pivot[0];
    hb.pivot[1] = b->pivot[1];
    hb.motion = b->motion;
    hb.x0[0] = b->x0[0];
    hb.x0[1] = b->x0[1];
    hb.alpha_mean = b->alpha_mean;
    hb.alpha_amp = b->alpha_amp;
    hb.period = b->period;
    hb.phase = b->phase;
    hb.heave_amp = b->heave_amp;
    hb.beta = b->stroke_beta;
    hb.u_ref = b->u_ref;
    hb.l_ref = b->l_ref;
    return true;
}

sbot_status sbot_set_body_kinematics(sbot_ctx_t c, const sbot_body_desc* b) {
    if (!c || !b) return SBOT_ERR_ARG;
    if (c->finalized && c->coarse_step > 0) return fail(c, SBOT_ERR_STATE, "set the body before stepping");
    HostBody& hb = c->body;
    if (!host_body_from_desc(b, hb)) return fail(c, SBOT_ERR_ARG, "bad body description");
    double R = 0;
    for (int j = 0; j < hb.n; j++)
        R = std::max(R, std::hypot(hb.qx[j] - hb.pivot[0], hb.qy[j] - hb.pivot[1]));
    hb.patch_side = (int)std::ceil(2 * R) + 6;
    int cap = hb.patch_side * hb.patch_side;
    size_t smem = ibm_smem_bytes(c->storage, cap, hb.n);
    if (smem > 220 * 1024) return fail(c, SBOT_ERR_ARG, "body too large for the one-block IBM kernel");
    c->ibm_smem = smem;
    c->has_body = true;
    InstParams& ip = c->ip;
    ip.has_body = 1;
    ip.n_markers = hb.n;
    ip.marker_off = 0;
    ip.ds = hb.ds;
    ip.pivot[0] = hb.pivot[0];
    ip.pivot[1] = hb.pivot[1];
    ip.motion = hb.motion;
    ip.x0[0] = hb.x0[0];
    ip.x0[1] = hb.x0[1];
    ip.alpha_mean = hb.alpha_mean;
    ip.alpha_amp = hb.alpha_amp;
    ip.period = hb.period;
    ip.phase = hb.phase;
    ip.heave_amp = hb.heave_amp;
    ip.beta = hb.beta;
    ip.cos_mean = std::cos(hb.alpha_mean);
    ip.sin_mean = std::sin(hb.alpha_mean);
    ip.patch_off = 0;
    ip.patch_cap = cap;
    dfree(c->d_qx);
    dfree(c->d_qy);
    dfree(c->d_patch);
    dfree(c->d_hist);
    CK(dalloc(&c->d_qx, hb.n));
    CK(dalloc(&c->d_qy, hb.n));
    CK(cudaMalloc(&c->d_patch, (size_t)2 * cap * (c->storage == 0 ? 8 : 4)));
    CK(dalloc(&c->d_hist, (size_t)3 * SBOT_HIST_CAP));
    CK(cudaMemcpyAsync(c->d_qx, hb.qx.data(), hb.n * sizeof(double), cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->d_qy, hb.qy.data(), hb.n * sizeof(double), cudaMemcpyHostToDevice, c->s));
    // rebuild the refinement around the body, drop the old state
    for (int sl = 0; sl < c->cap; sl++)
        if (c->h_type[sl] != ST_FREE) {
            c->h_type[sl] = ST_FREE;
            c->free_slots.push_back(sl);
        }
    c->bs = BlockStates();
    sbot_status st = build_topology(c, 0, false, nullptr);
    if (st != SBOT_OK) return st;
    return reset_state(c);
}

sbot_status sbot_set_fields(sbot_ctx_t c, int level, const double* rho, const double* ux, const double* uy) {
    if (!c || !rho || !ux || !uy) return SBOT_ERR_ARG;
    if (level_ok(c, level) != SBOT_OK) return SBOT_ERR_ARG;
    if (c->finalized) return fail(c, SBOT_ERR_STATE, "initial state can only be set before the first step");
    size_t plane = (size_t)(c->d.nx0 << level) * (c->d.ny0 << level);
    std::vector<double> tmp(3 * plane);
    std::memcpy(tmp.data(), rho, plane * sizeof(double));
    std::memcpy(tmp.data() + plane, ux, plane * sizeof(double));
    std::memcpy(tmp.data() + 2 * plane, uy, plane * sizeof(double));
    return upload_dense_pre(c, level, tmp.data(), 3, 1);
}

sbot_status sbot_set_populations(sbot_ctx_t c, int level, const double* f) {
    if (!c || !f) return SBOT_ERR_ARG;
    if (level_ok(c, level) != SBOT_OK) return SBOT_ERR_ARG;
    if (c->finalized) return fail(c, SBOT_ERR_STATE, "initial state can only be set before the first step");
    return upload_dense_pre(c, level, f, 9, 0);
}

sbot_status sbot_step(sbot_ctx_t c, int n) {
    if (!c || n < 0) return SBOT_ERR_ARG;
    sbot_status st = finalize_init(c);
    if (st != SBOT_OK) return st;
    const bool moving = c->d.retag && c->has_body;
    int k = 0;
    while (k < n) {
        if (!moving) {
            // static refinement: replay the coarse step from a CUDA graph.  Level
            // 0 flips its buffers once per coarse step, every finer level an even
            // number of times, so one graph per parity of level 0 covers all steps.
            int g = c->par[0];
            if (!c->gexec[g] || c->graph_version[g] != c->topo_version || c->graph_mask[g] != c->prof_mask) {
                CK(cudaStreamSynchronize(c->s));
                drop_graph(c, g);
                resolve_profile(c);
                int saved[SBOT_MAXLEV];
                std::memcpy(saved, c->par, sizeof saved);
                cudaGraph_t gr;
                c->capturing = true;
                CK(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
                DevPool P = pool_view(c);
                advance(c, P, 0);
                cudaError_t ce = cudaStreamEndCapture(c->s, &gr);
                c->capturing = false;
                CK(ce);
                c->graph_recs[g] = c->pending;
                c->pending.clear();
                std::memcpy(c->par, saved, sizeof saved);
                CK(cudaGraphInstantiate(&c->gexec[g], gr, 0));
                cudaGraphDestroy(gr);
                c->graph_version[g] = c->topo_version;
                c->graph_mask[g] = c->prof_mask;
            }
            CK(cudaGraphLaunch(c->gexec[g], c->s));
            if (c->prof_mask) resolve_graph_profile(c, g);
            c->par[0] ^= 1;
            c->coarse_step += 1;
            k += 1;
            continue;
        }
        if (moving && c->coarse_step > 0) {
            st = build_topology(c, c->coarse_step, true, nullptr);
            if (st != SBOT_OK) return st;
        }
        DevPool P = pool_view(c);
        advance(c, P, 0);
        c->coarse_step++;
        k++;
    }
    CK(cudaGetLastError());
    if (c->prof_mask) resolve_profile(c);
    return SBOT_OK;
}

sbot_status sbot_set_profiling(sbot_ctx_t c, int mask) {
    if (!c || mask < 0 || mask > 15) return SBOT_ERR_ARG;
    CK(cudaStreamSynchronize(c->s));
    resolve_profile(c);
    c->prof_mask = mask;
    if (mask)
        for (int k = 0; k < 4; k++) {
            c->prof_n[k] = 0;
            c->prof_ms[k] = 0;
            c->prof_bytes[k] = 0;
        }
    return SBOT_OK;
}

sbot_status sbot_get_profile(sbot_ctx_t c, int kind, int64_t* launches, double* ms, double* bytes) {
    if (!c || kind < 0 || kind > 3) return SBOT_ERR_ARG;
    resolve_profile(c);
    if (launches) *launches = c->prof_n[kind];
    if (ms) *ms = c->prof_ms[kind];
    if (bytes) *bytes = c->prof_bytes[kind];
    return SBOT_OK;
}

sbot_status sbot_get_forces(sbot_ctx_t c, double* fx, double* fy, double* mz, int* n_inout) {
    if (!c || !n_inout || *n_inout < 0) return SBOT_ERR_ARG;
    if (!c->has_body) {
        *n_inout = 0;
        return SBOT_OK;
    }
    sbot_status st = finalize_init(c);
    if (st != SBOT_OK) return st;
    CK(cudaStreamSynchronize(c->s));
    st = check_device_error(c);
    if (st != SBOT_OK) return st;
    long long upto = c->coarse_step << (c->m - 1);  // forces of finest steps k < canonical time
    long long avail = upto - c->forces_read;
    if (avail > SBOT_HIST_CAP) {
        c->forces_read = upto - SBOT_HIST_CAP;
        *n_inout = 0;
        return fail(c, SBOT_ERR_STATE, "force history overflowed; read forces more often");
    }
    int cnt = (int)std::min<long long>(avail, *n_inout);
    if (cnt > 0) {
        // the ring holds entry k at k mod capacity: at most two contiguous pieces
        std::vector<double> h((size_t)3 * cnt);
        long long k0 = c->forces_read % SBOT_HIST_CAP;
        long long first = std::min<long long>(cnt, SBOT_HIST_CAP - k0);
        CK(cudaMemcpy(h.data(), c->d_hist + 3 * k0, (size_t)3 * first * sizeof(double), cudaMemcpyDeviceToHost));
        if (first < cnt)
            CK(cudaMemcpy(h.data() + 3 * first, c->d_hist, (size_t)3 * (cnt - first) * sizeof(double),
                          cudaMemcpyDeviceToHost));
        for (int i = 0; i < cnt; i++) {
            if (fx) fx[i] = h[3 * i];
            if (fy) fy[i] = h[3 * i + 1];
            if (mz) mz[i] = h[3 * i + 2];
        }
    }
    c->forces_read += cnt;
    *n_inout = cnt;
    return SBOT_OK;
}

sbot_status sbot_get_fields(sbot_ctx_t c, int level, double* rho, double* ux, double* uy, int64_t* n_inout) {
    if (!c || !n_inout) return SBOT_ERR_ARG;
    if (level_ok(c, level) != SBOT_OK) return SBOT_ERR_ARG;
    int64_t plane = (int64_t)(c->d.nx0 << level) * (c->d.ny0 << level);
    if (*n_inout < plane) {
        *n_inout = plane;
        return fail(c, SBOT_ERR_ARG, "output arrays too small");
    }
    std::vector<double> out;
    sbot_status st = export_level(c, level, 1, out);
    if (st != SBOT_OK) return st;
    if (rho) std::memcpy(rho, out.data(), plane * sizeof(double));
    if (ux) std::memcpy(ux, out.data() + plane, plane * sizeof(double));
    if (uy) std::memcpy(uy, out.data() + 2 * plane, plane * sizeof(double));
    *n_inout = plane;
    return SBOT_OK;
}

sbot_status sbot_get_populations(sbot_ctx_t c, int level, double* f, int64_t* n_inout) {
    if (!c || !n_inout || !f) return SBOT_ERR_ARG;
    if (level_ok(c, level) != SBOT_OK) return SBOT_ERR_ARG;
    int64_t n = (int64_t)9 * (c->d.nx0 << level) * (c->d.ny0 << level);
    if (*n_inout < n) {
        *n_inout = n;
        return fail(c, SBOT_ERR_ARG, "output array too small");
    }
    std::vector<double> out;
    sbot_status st = export_level(c, level, 0, out);
    if (st != SBOT_OK) return st;
    std::memcpy(f, out.data(), n * sizeof(double));
    *n_inout = n;
    return SBOT_OK;
}

sbot_status sbot_get_celltypes(sbot_ctx_t c, int level, uint8_t* types, int64_t* n_inout) {
    if (!c || !n_inout || !types) return SBOT_ERR_ARG;
    if (level_ok(c, level) != SBOT_OK) return SBOT_ERR_ARG;
    std::vector<uint8_t> t;
    cell_types(c->ts, c->bs, level, t);
    if (*n_inout < (int64_t)t.size()) {
        *n_inout = (int64_t)t.size();
        return fail(c, SBOT_ERR_ARG, "output array too small");
    }
    std::memcpy(types, t.data(), t.size());
    *n_inout = (int64_t)t.size();
    return SBOT_OK;
}

sbot_status sbot_get_topology(sbot_ctx_t c, int level, uint8_t* states, int* n_inout) {
    if (!c || !n_inout || !states) return SBOT_ERR_ARG;
    if (level_ok(c, level) != SBOT_OK) return SBOT_ERR_ARG;
    const std::vector<uint8_t>& s = c->bs.s[level];
    if (*n_inout < (int)s.size()) {
        *n_inout = (int)s.size();
        return fail(c, SBOT_ERR_ARG, "output array too small");
    }
    std::memcpy(states, s.data(), s.size());
    *n_inout = (int)s.size();
    return SBOT_OK;
}

sbot_status sbot_get_checksum(sbot_ctx_t c, double out3[3]) {
    if (!c || !out3) return SBOT_ERR_ARG;
    sbot_status st = finalize_init(c);
    if (st != SBOT_OK) return st;
    DevPool P = pool_view(c);
    int total = 0;
    std::vector<int> nb(c->m);
    for (int l = 0; l < c->m; l++) {
        nb[l] = checksum_blocks(c->l_int[l].n, c->B);
        total += nb[l];
    }
    if (total > c->partials_cap) {
        dfree(c->d_partials);
        CK(dalloc(&c->d_partials, (size_t)3 * total));
        c->partials_cap = total;
    }
    bool direct = c->coarse_step == 0;
    int off = 0;
    for (int l = 0; l < c->m; l++) {
        double area = (double)(1LL << (2 * (c->m - 1 - l)));
        const void* src = direct ? c->f[1] : c->f[1 - c->par[l]];
        if (c->l_int[l].n > 0)
            launch_checksum_partials(c->storage, P, c->d_lists + c->l_int[l].off, c->l_int[l].n, src, l,
                                     direct ? 1 : 0, area, c->d_partials + 3 * off, nb[l], c->s);
        else
            CK(cudaMemsetAsync(c->d_partials + 3 * off, 0, 3 * nb[l] * sizeof(double), c->s));
        off += nb[l];
    }
    launch_reduce_partials(c->d_partials, total, c->d_out3, c->d_err, c->s);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out3, c->d_out3, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    return check_device_error(c);
}

// Same result as sbot_get_checksum, but allocates nothing: the partial sums
// go to the library's static device scratch instead of a buffer that
// sbot_get_checksum allocates on its first call.
sbot_status sbot_get_checksum_noalloc(sbot_ctx_t c, double out3[3]) {
    if (!c || !out3) return SBOT_ERR_ARG;
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != c->device) return fail(c, SBOT_ERR_STATE, "make the context's device current first");
    int total = 0;
    std::vector<int> nb(c->m);
    for (int l = 0; l < c->m; l++) {
        nb[l] = checksum_blocks(c->l_int[l].n, c->B);
        total += nb[l];
    }
    if (total > SBOT_NOALLOC_MAX_PARTIALS)
        return fail(c, SBOT_ERR_ARG,
                    "sbot_get_checksum_noalloc: this domain needs " + std::to_string(total) +
                        " partial sums; the static scratch holds " + std::to_string(SBOT_NOALLOC_MAX_PARTIALS) +
                        " (use sbot_get_checksum)");
    double* scratch = noalloc_scratch();
    if (!scratch) return fail(c, SBOT_ERR_CUDA, "cannot look up the static scratch on this device");
    sbot_status st = finalize_init(c);
    if (st != SBOT_OK) return st;
    DevPool P = pool_view(c);
    bool direct = c->coarse_step == 0;
    int off = 0;
    for (int l = 0; l < c->m; l++) {
        double area = (double)(1LL << (2 * (c->m - 1 - l)));
        const void* src = direct ? c->f[1] : c->f[1 - c->par[l]];
        if (c->l_int[l].n > 0)
            launch_checksum_partials(c->storage, P, c->d_lists + c->l_int[l].off, c->l_int[l].n, src, l,
                                     direct ? 1 : 0, area, scratch + 3 * off, nb[l], c->s);
        else
            CK(cudaMemsetAsync(scratch + 3 * off, 0, 3 * nb[l] * sizeof(double), c->s));
        off += nb[l];
    }
    double* res = scratch + 3 * SBOT_NOALLOC_MAX_PARTIALS;
    launch_reduce_partials(scratch, total, res, c->d_err, c->s);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out3, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    return check_device_error(c);
}

sbot_status sbot_get_level_info(sbot_ctx_t c, int level, int* nx, int* ny, int64_t* n_interior) {
    if (!c) return SBOT_ERR_ARG;
    if (level_ok(c, level) != SBOT_OK) return SBOT_ERR_ARG;
    if (nx) *nx = c->d.nx0 << level;
    if (ny) *ny = c->d.ny0 << level;
    if (n_interior) *n_interior = (int64_t)c->l_int[level].n * c->B * c->B;
    return SBOT_OK;
}

sbot_status sbot_get_work(sbot_ctx_t c, int64_t* cell_updates, int64_t* fine_equivalent) {
    if (!c) return SBOT_ERR_ARG;
    int64_t cu = 0;
    for (int l = 0; l < c->m; l++) cu += ((int64_t)c->l_int[l].n * c->B * c->B) << l;
    if (cell_updates) *cell_updates = cu;
    if (fine_equivalent)
        *fine_equivalent = ((int64_t)c->d.nx0 * c->d.ny0 << (2 * (c->m - 1))) << (c->m - 1);
    return SBOT_OK;
}

sbot_status sbot_plan_blocks(const sbot_domain_desc* desc, const sbot_body_desc* body, int64_t coarse_step,
                             int level, uint8_t* states, int* n_inout) {
    std::string why;
    if (!n_inout || !states || validate_desc(desc, why) != SBOT_OK) return SBOT_ERR_ARG;
    if (level < 0 || level >= desc->levels) return SBOT_ERR_ARG;
    sbot_ctx tmp;
    tmp.d = *desc;
    tmp.m = desc->levels;
    tmp.B = desc->block;
    for (int i = 0; i < desc->n_boxes; i++)
        tmp.static_boxes.push_back({desc->boxes[i].level, desc->boxes[i].x0, desc->boxes[i].y0, desc->boxes[i].x1,
                                    desc->boxes[i].y1});
    if (body) {
        if (!host_body_from_desc(body, tmp.body)) return SBOT_ERR_ARG;
        tmp.has_body = true;
    }
    TopoSpec ts;
    ts.m = tmp.m;
    ts.B = tmp.B;
    ts.nx0 = desc->nx0;
    ts.ny0 = desc->ny0;
    ts.periodic_x = desc->bc[SIDE_W] == BCK_PERIODIC;
    ts.periodic_y = desc->bc[SIDE_S] == BCK_PERIODIC;
    window_boxes(&tmp, coarse_step, ts.boxes);
    BlockStates bs;
    const char* w = nullptr;
    if (!plan_blocks(ts, bs, &w)) return SBOT_ERR_STATE;
    if (*n_inout < (int)bs.s[level].size()) {
        *n_inout = (int)bs.s[level].size();
        return SBOT_ERR_ARG;
    }
    std::memcpy(states, bs.s[level].data(), bs.s[level].size());
    *n_inout = (int)bs.s[level].size();
    return SBOT_OK;
}

sbot_status sbot_destroy(sbot_ctx_t c) {
    if (!c) return SBOT_OK;
    if (c->s) cudaStreamSynchronize(c->s);
    for (int i = 0; i < 2; i++) dfree(c->f[i]);
    void* ps[] = {c->d_nbr, c->d_inst, c->d_level, c->d_type, c->d_ox, c->d_oy, c->d_flags, c->d_parent, c->d_mask,
                  c->d_ip, c->d_ist, c->d_latmap, c->d_qx, c->d_qy, c->d_patch, c->d_hist, c->d_err, c->d_lists,
                  c->d_ibm_list, c->d_partials, c->d_out3};
    for (void* p : ps) dfree(p);
    for (int g = 0; g < 2; g++) drop_graph(c, g);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (int l = 0; l < SBOT_MAXLEV; l++) {
        if (c->side[l]) cudaStreamSynchronize(c->side[l]);
        if (c->side[l]) cudaStreamDestroy(c->side[l]);
        if (c->ev_fork[l]) cudaEventDestroy(c->ev_fork[l]);
        if (c->ev_join[l]) cudaEventDestroy(c->ev_join[l]);
    }
    if (c->own_stream) cudaStreamDestroy(c->s);
    delete c;
    return SBOT_OK;
}

const char* sbot_last_error(sbot_ctx_t c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
