// Host emulation of the GPU labelling path, for tests only.
//
// It compiles the very same tile phases (paper_1606_05973_gb300/csrc/ccl_core.cuh) with a
// host C++ compiler and runs every CTA's threads one after another within each phase, in
// a seeded random order, with the shared-memory tile poisoned before use.  Built with
// AddressSanitizer it checks the kernels' index arithmetic and the absence of reads of
// unwritten shared memory on the CPU, before anything runs on a GPU.  The library never
// loads this file; it is not a way to label images in production.
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <random>
#include <vector>

#include "../../paper_1606_05973_gb300/csrc/ccl_core.cuh"

using namespace ccl;

namespace {

template <class C> struct Emu {
    std::mt19937_64 rng;
    std::vector<int> order;

    explicit Emu(uint64_t seed) : rng(seed), order(C::NT) { std::iota(order.begin(), order.end(), 0); }

    template <class F> void phase(F f)
    {
        std::shuffle(order.begin(), order.end(), rng);
        for (int t : order)
            f(t);
    }

    int64_t run(const uint8_t *img, int H, int W, int64_t pitch, int32_t *labels, int32_t *status)
    {
        if (H == 0 || W == 0)
            return 0;
        const Layout L = plan_layout<C>(H, W);
        std::vector<unsigned char> ws((size_t)L.bytes + 64);
        // poison the workspace: every value the kernels read must have been written
        memset(ws.data(), 0x7B, ws.size());
        int K = -1;
        Img a;
        memset(&a, 0, sizeof(a));
        a.img = img;
        a.pitch = pitch;
        a.H = H;
        a.W = W;
        a.vec_in = ((uintptr_t)img % 16 == 0) && (pitch % 16 == 0);
        a.labels = labels;
        a.vec_out = ((uintptr_t)labels % 16 == 0) && (W % 4 == 0);
        a.K = &K;
        a.status = status;
        char *b = (char *)ws.data();
        a.nTX = L.nTX;
        a.nTY = L.nTY;
        a.bitpack = (uint32_t *)(b + L.off_bitpack);
        a.runinfo = (uint16_t *)(b + L.off_runinfo);
        a.nRunInfo = L.nRunInfo;
        a.P = (int *)(b + L.off_P);
        a.nseg = (int *)(b + L.off_nseg);
        a.cnt = (int *)(b + L.off_cnt);
        a.edgeRow = (int *)(b + L.off_edgeRow);
        a.edgeCol = (int *)(b + L.off_edgeCol);
        a.bsum = (int *)(b + L.off_bsum);
        a.nP = L.nP;
        a.nSeg = L.nSeg;

        const int ntiles = L.nTX * L.nTY;
        std::vector<int> tiles(ntiles);
        std::iota(tiles.begin(), tiles.end(), 0);
        auto *s = new SmemL<C>;
        auto *f = new SmemF<C>;
        using T = Tile<C>;

        // tile_local
        std::shuffle(tiles.begin(), tiles.end(), rng);
        for (int tile : tiles) {
            const int ty = tile / a.nTX, tx = tile % a.nTX;
            memset(s, 0x7F, sizeof(*s));
            phase([&](int t) { T::load_image(a, *s, ty, tx, t); });
            phase([&](int t) { T::store_bitpack(a, *s, ty, tx, t); T::strip_runs(*s, t); });
            phase([&](int t) { T::strip_prefix(*s, t); });
            phase([&](int t) { T::unions(a, *s, t); });
            phase([&](int t) { T::roots(a, *s, t); });
            phase([&](int t) { T::first_pixels(a, *s, t); });
            phase([&](int t) { T::mark_roots(a, *s, t); });
            phase([&](int t) { T::root_prefix(a, *s, ty, tx, t); });
            phase([&](int t) { T::outputs(a, *s, ty, tx, t); });
        }
        // boundary merge, items in random order
        {
            const int64_t nh = (int64_t)(a.nTY - 1) * a.W, nv = (int64_t)(a.nTX - 1) * a.H;
            std::vector<int64_t> items(nh + nv);
            std::iota(items.begin(), items.end(), 0);
            std::shuffle(items.begin(), items.end(), rng);
            for (int64_t i : items) {
                if (i < nh)
                    merge_h<C>(a, 1 + (int)(i / a.W), (int)(i % a.W));
                else
                    merge_v<C>(a, 1 + (int)((i - nh) / a.H), (int)((i - nh) % a.H));
            }
        }
        // flatten: rounds of pointer jumping over the segments (random order) until a
        // round leaves every node at its root, as the cooperative kernel does
        {
            std::vector<int64_t> segs(L.nSeg);
            std::iota(segs.begin(), segs.end(), 0);
            for (int r = 0; r < MAX_ROUNDS; r++) {
                std::shuffle(segs.begin(), segs.end(), rng);
                bool more = false;
                for (int64_t sg : segs)
                    more |= jump_segment<C>(a, sg);
                if (!more)
                    break;
                if (r == MAX_ROUNDS - 1)
                    *a.status |= ST_LOOP_CAP;
            }
        }
        // root count, scan and labels with a pseudo-grid of G CTAs of GNT threads
        {
            const int G = (int)std::min<int64_t>(3, (L.nSeg + GNT - 1) / GNT);
            std::vector<int> tot(G), excl((size_t)G * GNT), cnt((size_t)G * GNT);
            for (int bb = 0; bb < G; bb++) {
                ScanBuf sb;
                for (int t = 0; t < GNT; t++) {
                    int64_t s0, s1;
                    seg_range(L.nSeg, G, GNT, bb, t, &s0, &s1);
                    cnt[(size_t)bb * GNT + t] = count_roots<C>(a, s0, s1);
                    scan_put(sb, t, cnt[(size_t)bb * GNT + t]);
                }
                for (int k = 0; k < GNT_LOG; k++)
                    for (int t = 0; t < GNT; t++)
                        scan_step(sb, t, k);
                for (int t = 0; t < GNT; t++)
                    excl[(size_t)bb * GNT + t] = scan_incl(sb, t) - cnt[(size_t)bb * GNT + t];
                tot[bb] = scan_incl(sb, GNT - 1);
            }
            int acc = 0;
            for (int bb = 0; bb < G; bb++) {
                const int t = tot[bb];
                tot[bb] = acc;
                acc += t;
            }
            *a.K = acc;
            for (int bb = 0; bb < G; bb++)
                for (int t = 0; t < GNT; t++) {
                    int64_t s0, s1;
                    seg_range(L.nSeg, G, GNT, bb, t, &s0, &s1);
                    label_roots<C>(a, s0, s1, tot[bb] + excl[(size_t)bb * GNT + t]);
                }
        }
        std::shuffle(tiles.begin(), tiles.end(), rng);
        for (int tile : tiles) {
            const int ty = tile / a.nTX, tx = tile % a.nTX;
            memset(f, 0x7F, sizeof(*f));
            phase([&](int t) { T::load_bitpack(a, *f, ty, tx, t); });
            phase([&](int t) { T::strip_runs(*f, t); });
            phase([&](int t) { T::strip_prefix(*f, t); });
            phase([&](int t) { T::run_labels(a, *f, ty, tx, t); });
            phase([&](int t) { T::write_labels(a, *f, ty, tx, t); });
        }
        delete s;
        delete f;
        return K;
    }
};

}  // namespace

extern "C" {

// shapes: 0 = the library's main tile (64x256, 256 threads); 1 = small tile (4x32, 32 threads)
int64_t emu_label(const uint8_t *img, int32_t H, int32_t W, int64_t pitch, int32_t *labels,
                  uint64_t seed, int32_t shape, int32_t *status)
{
    *status = 0;
    if (shape == 0) {
        Emu<Cfg<64, 256, 256>> e(seed);
        return e.run(img, H, W, pitch, labels, status);
    } else if (shape == 1) {
        Emu<Cfg<4, 32, 32>> e(seed);
        return e.run(img, H, W, pitch, labels, status);
    } else {
        Emu<Cfg<8, 64, 64>> e(seed);
        return e.run(img, H, W, pitch, labels, status);
    }
}

}  // extern "C"
