// Spatial tiles of a burst for independent processes (one per GPU or per
// job): output pixels depend only on the samples in their SHP window, so a
// burst splits into tiles of output cells, each processed from an input crop
// that holds its cells' windows (a read-only halo, no exchange).  Along a
// sequential chain the compressed SLC of a mini-stack enters the next one's
// windows, so each further step needs one more window of halo (the dependency
// cone).  Host code only.
//
// Exactness, per axis (rows and columns separate: a window is a product of a
// row and a column interval, and so is everything derived from it).  A crop
// [c0, c1) with c0 a multiple of the stride s has cells whose centres are the
// burst's (c0 + j s + s/2 = (c0/s + j) s + s/2).  Burst cell i is exact at
// step 1 when it is one of the crop's cells, its window clipped to the burst
// lies inside the crop (so the crop clips it the same way), and its
// decimation block -- which the compressed SLC and the PS regridding use, the
// last cell's running to the image end -- is the same in the crop and in the
// burst.  At a later step it also needs every row of its window to carry an
// exact compressed SLC from every earlier step, i.e. each such row's cell to
// have been exact there.  The plan takes, for each tile, the smallest crop
// (grown a stride at a time on both sides, clipped to the burst) whose owned
// cells are exact at every step.
#include <string.h>

#include <vector>

#include "api_internal.h"

using namespace plkapi;

namespace {

struct Axis {
    int L, s, h;  // image length, stride, half window
    int G() const { return L / s; }
    int block_lo(int i) const { return i * s; }
    int block_hi(int i) const { return (i == G() - 1) ? L : (i + 1) * s; }
};

// Cells [a, b) of the burst exact at every one of `steps` steps on crop [c0, c1)?
bool exact(const Axis &ax, int c0, int c1, int a, int b, int steps) {
    const int G = ax.G();
    const int first = c0 / ax.s, Gc = (c1 - c0) / ax.s;  // crop cells: burst cells first .. first + Gc - 1
    if (a < first || b > first + Gc) return false;
    // exactness of the crop's cells (index i - first); a cell outside the crop is never exact
    std::vector<char> prev(Gc, 0), cur(Gc, 0);
    for (int step = 1; step <= steps; ++step) {
        for (int j = 0; j < Gc; ++j) {
            const int i = first + j;
            cur[j] = 0;
            const int crop_hi = (j == Gc - 1) ? c1 : c0 + (j + 1) * ax.s;
            if (ax.block_lo(i) != c0 + j * ax.s || ax.block_hi(i) != crop_hi) continue;
            const int centre = i * ax.s + ax.s / 2;
            const int w0 = centre - ax.h < 0 ? 0 : centre - ax.h;
            const int w1 = centre + ax.h + 1 > ax.L ? ax.L : centre + ax.h + 1;
            if (w0 < c0 || w1 > c1) continue;
            bool ok = true;
            if (step > 1)
                for (int y = w0; y < w1 && ok; ++y) {
                    const int cell = (y / ax.s < G - 1) ? y / ax.s : G - 1;
                    ok = cell >= first && cell < first + Gc && prev[cell - first] != 0;
                }
            cur[j] = ok ? 1 : 0;
        }
        for (int i = a; i < b; ++i)
            if (!cur[i - first]) return false;
        // a compressed SLC row is exact after this step and all earlier ones;
        // once that set stops changing, every later step repeats this one
        bool changed = step == 1;
        for (int j = 0; j < Gc; ++j) {
            const char v = (step == 1 ? cur[j] : (prev[j] && cur[j])) ? 1 : 0;
            changed = changed || v != prev[j];
            prev[j] = v;
        }
        if (!changed) break;
    }
    return true;
}

// The smallest crop, grown one stride at a time on both sides, for cells
// [a, b).  A larger crop keeps every cell a smaller one makes exact, so the
// margin is found by bisection; the whole axis is always exact.
void plan_axis(const Axis &ax, int a, int b, int steps, int *c0, int *c1) {
    const int lo0 = ax.block_lo(a), hi0 = ax.block_hi(b - 1);
    auto crop = [&](int m, int *lo, int *hi) {
        *lo = lo0 - m * ax.s < 0 ? 0 : lo0 - m * ax.s;
        *hi = hi0 + m * ax.s > ax.L ? ax.L : hi0 + m * ax.s;
    };
    int m_lo = 0, m_hi = (lo0 + ax.s - 1) / ax.s;
    if ((ax.L - hi0 + ax.s - 1) / ax.s > m_hi) m_hi = (ax.L - hi0 + ax.s - 1) / ax.s;
    while (m_lo < m_hi) {  // smallest m in [m_lo, m_hi] whose crop is exact
        const int m = (m_lo + m_hi) / 2;
        int lo, hi;
        crop(m, &lo, &hi);
        if (exact(ax, lo, hi, a, b, steps)) m_hi = m;
        else m_lo = m + 1;
    }
    crop(m_lo, c0, c1);
}

}  // namespace

extern "C" {

plk_status plk_tile_plan(int H, int W, plk_window win, int tiles_y, int tiles_x, int steps, plk_tile *tiles) {
    if (!tiles || H < 1 || W < 1 || !window_ok(win) || steps < 1 || steps > 256)
        return fail(nullptr, PLK_EINVAL, "plk_tile_plan: bad argument");
    const Axis ay{H, win.sy, win.wy / 2}, ax{W, win.sx, win.wx / 2};
    if (tiles_y < 1 || tiles_x < 1 || tiles_y > ay.G() || tiles_x > ax.G())
        return fail(nullptr, PLK_EINVAL, "plk_tile_plan: %d x %d tiles of a %d x %d output grid", tiles_y, tiles_x,
                    ay.G(), ax.G());
    std::vector<int> ry(2 * tiles_y), rx(2 * tiles_x);
    for (int t = 0; t < tiles_y; ++t) {
        const int a = (int)((long long)t * ay.G() / tiles_y), b = (int)((long long)(t + 1) * ay.G() / tiles_y);
        plan_axis(ay, a, b, steps, &ry[2 * t], &ry[2 * t + 1]);
    }
    for (int t = 0; t < tiles_x; ++t) {
        const int a = (int)((long long)t * ax.G() / tiles_x), b = (int)((long long)(t + 1) * ax.G() / tiles_x);
        plan_axis(ax, a, b, steps, &rx[2 * t], &rx[2 * t + 1]);
    }
    for (int ty = 0; ty < tiles_y; ++ty)
        for (int tx = 0; tx < tiles_x; ++tx) {
            plk_tile &T = tiles[ty * tiles_x + tx];
            memset(&T, 0, sizeof(T));
            const int a_y = (int)((long long)ty * ay.G() / tiles_y), b_y = (int)((long long)(ty + 1) * ay.G() / tiles_y);
            const int a_x = (int)((long long)tx * ax.G() / tiles_x), b_x = (int)((long long)(tx + 1) * ax.G() / tiles_x);
            T.y0 = ry[2 * ty];
            T.h = ry[2 * ty + 1] - T.y0;
            T.x0 = rx[2 * tx];
            T.w = rx[2 * tx + 1] - T.x0;
            T.oy0 = a_y;
            T.oh = b_y - a_y;
            T.ox0 = a_x;
            T.ow = b_x - a_x;
            T.cy0 = a_y - T.y0 / win.sy;
            T.cx0 = a_x - T.x0 / win.sx;
            T.py0 = ay.block_lo(a_y);
            T.ph = ay.block_hi(b_y - 1) - T.py0;
            T.px0 = ax.block_lo(a_x);
            T.pw = ax.block_hi(b_x - 1) - T.px0;
        }
    return PLK_OK;
}

}  // extern "C"
