// Host-side planning of the block-refined grid (Sec. 2.3-2.4 of arXiv 2402.04606).
#pragma once
#include <cstdint>
#include <vector>

struct RefBox {
    int level;
    double x0, y0, x1, y1;  // finest units, open rectangle
};

struct TopoSpec {
    int m, B, nx0, ny0;
    bool periodic_x, periodic_y;
    std::vector<RefBox> boxes;  // static boxes plus the body boxes of the current window
};

// block states per level: 0 absent (inside a coarser leaf), 1 leaf, 2 refined
struct BlockStates {
    std::vector<int> nbx, nby;
    std::vector<std::vector<uint8_t>> s;
    uint8_t at(int l, int bx, int by) const { return s[l][(size_t)by * nbx[l] + bx]; }
};

// refine every leaf that meets a box of a finer level, then enforce the 2:1
// balance over faces and corners; returns false (and a message) when the
// refinement touches a non-periodic side
bool plan_blocks(const TopoSpec& t, BlockStates& out, const char** why);

// one block of a level that needs a slot
struct PlannedBlock {
    int level, bx, by;
    int type;  // ST_INT / ST_GF / ST_GC
    std::vector<uint32_t> mask;  // halo (GF, within 2 cells of the interior) or mailbox (GC, within 1 cell)
};

// all blocks that need storage, level by level, in lattice order
void plan_slots(const TopoSpec& t, const BlockStates& bs, std::vector<PlannedBlock>& out);

// dense cell kinds of one level (0 none, 1 interior, 2 halo, 3 mailbox)
void cell_types(const TopoSpec& t, const BlockStates& bs, int level, std::vector<uint8_t>& out);
