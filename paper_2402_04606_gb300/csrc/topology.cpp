// Host-side planning of the block-refined grid: topology-confined block
// refinement (Sec. 2.3), level jump of at most one between blocks that share
// a face or a corner and two halo layers (Sec. 2.4).
#include "topology.h"

#include <algorithm>

#include "sbot_internal.h"

namespace {

bool wrap_block(int v, int n, bool periodic, int& out) {
    if (v >= 0 && v < n) {
        out = v;
        return true;
    }
    if (!periodic) return false;
    out = ((v % n) + n) % n;
    return true;
}

void split(const TopoSpec& t, BlockStates& bs, int l, int bx, int by) {
    bs.s[l][(size_t)by * bs.nbx[l] + bx] = 2;
    for (int j = 0; j < 2; j++)
        for (int i = 0; i < 2; i++) bs.s[l + 1][(size_t)(2 * by + j) * bs.nbx[l + 1] + 2 * bx + i] = 1;
}

}  // namespace

bool plan_blocks(const TopoSpec& t, BlockStates& bs, const char** why) {
    bs.nbx.assign(t.m, 0);
    bs.nby.assign(t.m, 0);
    bs.s.assign(t.m, {});
    for (int l = 0; l < t.m; l++) {
        bs.nbx[l] = (t.nx0 << l) / t.B;
        bs.nby[l] = (t.ny0 << l) / t.B;
        bs.s[l].assign((size_t)bs.nbx[l] * bs.nby[l], 0);
    }
    std::fill(bs.s[0].begin(), bs.s[0].end(), 1);
    // a level-l block [X0, X1) x [Y0, Y1) (finest units) is split when it meets
    // a region that asks for level l+1 or finer
    for (int l = 0; l + 1 < t.m; l++) {
        double side = (double)t.B * (double)(1 << (t.m - 1 - l));
        for (int by = 0; by < bs.nby[l]; by++)
            for (int bx = 0; bx < bs.nbx[l]; bx++) {
                if (bs.at(l, bx, by) != 1) continue;
                double X0 = bx * side, X1 = X0 + side, Y0 = by * side, Y1 = Y0 + side;
                bool hit = false;
                for (const RefBox& r : t.boxes)
                    if (r.level > l && X0 < r.x1 && r.x0 < X1 && Y0 < r.y1 && r.y0 < Y1) hit = true;
                if (hit) split(t, bs, l, bx, by);
            }
    }
    // 2:1 balance: a leaf must not touch a split block of the next level
    for (bool again = true; again;) {
        again = false;
        for (int l = 0; l + 2 < t.m; l++)
            for (int by = 0; by < bs.nby[l]; by++)
                for (int bx = 0; bx < bs.nbx[l]; bx++) {
                    if (bs.at(l, bx, by) != 1) continue;
                    bool touch = false;
                    for (int j = 2 * by - 1; j <= 2 * by + 2 && !touch; j++)
                        for (int i = 2 * bx - 1; i <= 2 * bx + 2 && !touch; i++) {
                            if (i >= 2 * bx && i < 2 * bx + 2 && j >= 2 * by && j < 2 * by + 2) continue;
                            int wi, wj;
                            if (!wrap_block(i, bs.nbx[l + 1], t.periodic_x, wi)) continue;
                            if (!wrap_block(j, bs.nby[l + 1], t.periodic_y, wj)) continue;
                            touch = bs.at(l + 1, wi, wj) == 2;
                        }
                    if (touch) {
                        split(t, bs, l, bx, by);
                        again = true;
                    }
                }
    }
    for (int l = 1; l < t.m; l++)
        for (int by = 0; by < bs.nby[l]; by++)
            for (int bx = 0; bx < bs.nbx[l]; bx++) {
                if (bs.at(l, bx, by) == 0) continue;
                bool edge = (!t.periodic_x && (bx == 0 || bx == bs.nbx[l] - 1)) ||
                            (!t.periodic_y && (by == 0 || by == bs.nby[l] - 1));
                if (edge) {
                    *why = "refinement touches a non-periodic domain side";
                    return false;
                }
            }
    return true;
}

void plan_slots(const TopoSpec& t, const BlockStates& bs, std::vector<PlannedBlock>& out) {
    out.clear();
    const int B = t.B;
    const int words = (B * B + 31) / 32;
    for (int l = 0; l < t.m; l++)
        for (int by = 0; by < bs.nby[l]; by++)
            for (int bx = 0; bx < bs.nbx[l]; bx++) {
                int st = bs.at(l, bx, by);
                PlannedBlock pb;
                pb.level = l;
                pb.bx = bx;
                pb.by = by;
                pb.mask.assign(words, 0u);
                if (st == 1) {
                    pb.type = ST_INT;
                    std::fill(pb.mask.begin(), pb.mask.end(), 0xffffffffu);
                    out.push_back(pb);
                    continue;
                }
                // halo (inside a coarser leaf) reaches 2 cells, mailbox (inside the finer region) 1 cell
                int reach = (st == 0) ? 2 : 1;
                bool any = false;
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        if (!dx && !dy) continue;
                        int nx, ny;
                        if (!wrap_block(bx + dx, bs.nbx[l], t.periodic_x, nx)) continue;
                        if (!wrap_block(by + dy, bs.nby[l], t.periodic_y, ny)) continue;
                        if (bs.at(l, nx, ny) != 1) continue;
                        for (int y = 0; y < B; y++)
                            for (int x = 0; x < B; x++) {
                                int ex = dx > 0 ? B - x : (dx < 0 ? x + 1 : 0);
                                int ey = dy > 0 ? B - y : (dy < 0 ? y + 1 : 0);
                                if (std::max(ex, ey) <= reach) {
                                    int c = y * B + x;
                                    pb.mask[c >> 5] |= 1u << (c & 31);
                                    any = true;
                                }
                            }
                    }
                if (!any) continue;
                pb.type = (st == 0) ? ST_GF : ST_GC;
                out.push_back(pb);
            }
}

void cell_types(const TopoSpec& t, const BlockStates& bs, int level, std::vector<uint8_t>& out) {
    const int B = t.B;
    int nx = t.nx0 << level, ny = t.ny0 << level;
    out.assign((size_t)nx * ny, 0);
    std::vector<PlannedBlock> pbs;
    plan_slots(t, bs, pbs);
    for (const PlannedBlock& pb : pbs) {
        if (pb.level != level) continue;
        for (int y = 0; y < B; y++)
            for (int x = 0; x < B; x++) {
                int c = y * B + x;
                if (!((pb.mask[c >> 5] >> (c & 31)) & 1u)) continue;
                out[(size_t)(pb.by * B + y) * nx + pb.bx * B + x] = (uint8_t)pb.type;
            }
    }
}
