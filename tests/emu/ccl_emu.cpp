// Host emulation of the GPU labelling path, for tests only.
//
// It compiles the very same kernel bodies (paper_1606_05973_gb300/csrc/ccl_core.cuh) with
// a host C++ compiler and runs each CUDA thread as a fiber:
//   __syncthreads()        -> a barrier over the CTA's fibers
//   warp shuffle / ballot  -> a per-warp exchange slot between two warp barriers
//   atomics                -> a point where the scheduler may switch to another fiber
//   cooperative grid sync  -> a barrier over every fiber of every CTA
// Shared memory and the workspace are poisoned before use, and the bounds-checked build
// is on, so under AddressSanitizer any out-of-range access or read of unwritten memory in
// the kernels fails here, on the CPU, before anything runs on a GPU.  The library never
// loads this file; it is not a way to label images in production.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <ucontext.h>

#include <algorithm>
#include <array>
#include <functional>
#include <memory>
#include <numeric>
#include <random>
#include <vector>

#include "../../paper_1606_05973_gb300/csrc/ccl_core.cuh"

#if defined(__SANITIZE_ADDRESS__)
#define EMU_ASAN 1
extern "C" void __sanitizer_start_switch_fiber(void **fake_stack_save, const void *bottom, size_t size);
extern "C" void __sanitizer_finish_switch_fiber(void *fake_stack_save, const void **bottom_old, size_t *size_old);
#endif

using namespace ccl;

namespace {

// Every emulated CUDA thread is a fiber (ucontext) on the calling OS thread.  A seeded
// scheduler picks which runnable fiber continues whenever one blocks on a barrier or
// reaches an atomic (emu_yield), so different seeds give different interleavings.  If no
// fiber can run and some are unfinished (a barrier that not every thread reaches, e.g. a
// divergent warp shuffle) the emulator aborts instead of hanging.
struct Barrier {
    int expected = 0, arrived = 0;
    std::vector<int> waiting;
};

struct Fib {
    ucontext_t ctx;
    std::unique_ptr<char[]> stack;
    int cta = 0, tid = 0;
    bool done = false, runnable = true;
};

constexpr size_t kStack = 256 * 1024;

struct Sched {
    std::vector<Fib> fibs;
    ucontext_t main_ctx;
    int cur = -1;
    std::mt19937_64 rng;
    std::vector<Barrier> cta_bar;
    std::vector<std::vector<Barrier>> warp_bar;
    std::vector<std::vector<std::array<uint32_t, 32>>> slot;
    Barrier grid_bar;
    std::function<void(int, int)> body;
#if defined(EMU_ASAN)
    const void *main_bottom = nullptr;
    size_t main_size = 0;
#endif

    Sched(int nctas, int nt, uint64_t seed, std::function<void(int, int)> f) : rng(seed), body(std::move(f))
    {
        const int nw = (nt + 31) / 32;
        cta_bar.resize(nctas);
        warp_bar.resize(nctas);
        slot.resize(nctas);
        for (int c = 0; c < nctas; c++) {
            cta_bar[c].expected = nt;
            warp_bar[c].resize(nw);
            for (int w = 0; w < nw; w++)
                warp_bar[c][w].expected = (w == nw - 1 && nt % 32) ? nt % 32 : 32;
            slot[c].resize(nw);
        }
        grid_bar.expected = nctas * nt;
        fibs.resize((size_t)nctas * nt);
        for (int c = 0; c < nctas; c++)
            for (int t = 0; t < nt; t++) {
                Fib &f = fibs[(size_t)c * nt + t];
                f.cta = c;
                f.tid = t;
            }
    }

    void to_main()
    {
#if defined(EMU_ASAN)
        void *fake = nullptr;
        __sanitizer_start_switch_fiber(&fake, main_bottom, main_size);
#endif
        swapcontext(&fibs[cur].ctx, &main_ctx);
#if defined(EMU_ASAN)
        __sanitizer_finish_switch_fiber(fake, nullptr, nullptr);
#endif
    }

    void arrive(Barrier &b)
    {
        b.arrived++;
        if (b.arrived == b.expected) {
            for (int f : b.waiting)
                fibs[f].runnable = true;
            b.waiting.clear();
            b.arrived = 0;
            to_main();  // let the scheduler pick who goes on
        } else {
            b.waiting.push_back(cur);
            fibs[cur].runnable = false;
            to_main();
        }
    }

    static void trampoline(int hi, int lo);

    void run()
    {
        for (size_t i = 0; i < fibs.size(); i++) {
            Fib &f = fibs[i];
            f.stack.reset(new char[kStack]);
            getcontext(&f.ctx);
            f.ctx.uc_stack.ss_sp = f.stack.get();
            f.ctx.uc_stack.ss_size = kStack;
            f.ctx.uc_link = &main_ctx;
            const uintptr_t self = reinterpret_cast<uintptr_t>(this);
            makecontext(&f.ctx, (void (*)())trampoline, 2, (int)(self >> 32), (int)(self & 0xFFFFFFFFu));
        }
        std::vector<int> ready;
        for (;;) {
            ready.clear();
            bool all_done = true;
            for (size_t i = 0; i < fibs.size(); i++) {
                if (!fibs[i].done) {
                    all_done = false;
                    if (fibs[i].runnable)
                        ready.push_back((int)i);
                }
            }
            if (all_done)
                return;
            if (ready.empty()) {
                fprintf(stderr, "emulator deadlock: a barrier or warp collective not reached by every thread\n");
                abort();
            }
            cur = ready[rng() % ready.size()];
#if defined(EMU_ASAN)
            void *fake = nullptr;
            __sanitizer_start_switch_fiber(&fake, fibs[cur].stack.get(), kStack);
#endif
            swapcontext(&main_ctx, &fibs[cur].ctx);
#if defined(EMU_ASAN)
            __sanitizer_finish_switch_fiber(fake, &main_bottom, &main_size);
#endif
        }
    }
};

Sched *g_sched = nullptr;

void Sched::trampoline(int hi, int lo)
{
    Sched *s = reinterpret_cast<Sched *>(((uintptr_t)(uint32_t)hi << 32) | (uintptr_t)(uint32_t)lo);
#if defined(EMU_ASAN)
    __sanitizer_finish_switch_fiber(nullptr, &s->main_bottom, &s->main_size);
#endif
    const int me = s->cur;
    s->body(s->fibs[me].cta, s->fibs[me].tid);
    s->fibs[me].done = true;
#if defined(EMU_ASAN)
    void *fake = nullptr;
    __sanitizer_start_switch_fiber(&fake, s->main_bottom, s->main_size);
#endif
    // returning resumes main_ctx through uc_link
}

Fib &me() { return g_sched->fibs[g_sched->cur]; }

}  // namespace

void emu_cta_sync() { g_sched->arrive(g_sched->cta_bar[me().cta]); }
void emu_grid_sync() { g_sched->arrive(g_sched->grid_bar); }
void emu_yield()
{
    if ((g_sched->rng() & 3) == 0)
        g_sched->to_main();
}
int emu_lane() { return me().tid & 31; }

static uint32_t *warp_slots() { return g_sched->slot[me().cta][me().tid / 32].data(); }
static void warp_sync_emu() { g_sched->arrive(g_sched->warp_bar[me().cta][me().tid / 32]); }

uint32_t emu_ballot(bool p)
{
    uint32_t *sl = warp_slots();
    const int l = me().tid & 31;
    sl[l] = p ? 1u : 0u;
    warp_sync_emu();
    uint32_t m = 0;
    for (int i = 0; i < 32; i++)
        m |= (sl[i] & 1u) << i;
    warp_sync_emu();
    return m;
}
int emu_shfl(int v, int src, int width)
{
    uint32_t *sl = warp_slots();
    const int l = me().tid & 31;
    sl[l] = (uint32_t)v;
    warp_sync_emu();
    const int r = (int)sl[(l & ~(width - 1)) + (src & (width - 1))];
    warp_sync_emu();
    return r;
}
int emu_shfl_up(int v, int delta, int width)
{
    uint32_t *sl = warp_slots();
    const int l = me().tid & 31;
    sl[l] = (uint32_t)v;
    warp_sync_emu();
    const int r = ((l & (width - 1)) >= delta) ? (int)sl[l - delta] : v;
    warp_sync_emu();
    return r;
}

namespace {

int g_emu_thr = 0;  // object = byte > g_emu_thr

template <class C> struct Emu {
    uint64_t seed;
    std::mt19937_64 rng;

    explicit Emu(uint64_t s) : seed(s), rng(s) {}

    // NT threads of one persistent CTA walk every tile (in a shuffled order)
    template <class Smem, class Body> void run_tiles(int ntiles, Body body)
    {
        std::vector<int> order(ntiles);
        std::iota(order.begin(), order.end(), 0);
        std::shuffle(order.begin(), order.end(), rng);
        auto smem = std::make_unique<Smem>();
        Sched sch(1, C::NT, rng(), [&](int, int t) {
            for (int tile : order) {
                if (t == 0)
                    memset(smem.get(), 0x7F, sizeof(Smem));
                emu_cta_sync();
                body(*smem, tile, t);
                emu_cta_sync();
            }
        });
        g_sched = &sch;
        sch.run();
        g_sched = nullptr;
    }

    // G CTAs of NTG threads, all running at once (cooperative launch)
    template <int NTG = GNT> void run_global(const Img &a, int G)
    {
        std::vector<ScanBufT<NTG>> sbs(G);
        std::vector<int> flags(G);
        Sched sch(G, NTG, rng(), [&](int b, int t) { global_body<C, NTG>(a, sbs[b], flags[b], b, G, t); });
        g_sched = &sch;
        sch.run();
        g_sched = nullptr;
    }

    // the batched kernels over n images (all with H, W > 0), as ccl_label_batch runs them
    void run_batch(int n, const uint8_t *const *imgs, const int32_t *Hs, const int32_t *Ws, const int64_t *pitches,
                   int32_t *const *labels, int32_t *Ks, int32_t *status)
    {
        std::vector<Layout> L(n);
        std::vector<std::vector<unsigned char>> ws(n);
        std::vector<Img> descs(n);
        std::vector<int64_t> tileStart(n + 1), itemStart(n + 1), segStart(n + 1);
        std::vector<int> imgBase(n + 1, 0x7B7B7B7B), bsum(MAX_GLOBAL_CTAS, 0x7B7B7B7B);
        std::vector<unsigned char> hdr(256, 0x7B);
        for (int i = 0; i < n; i++) {
            L[i] = plan_layout<C>(Hs[i], Ws[i]);
            ws[i].assign((size_t)L[i].bytes + 64, 0x7B);
            Img &a = descs[i];
            memset(&a, 0, sizeof(a));
            a.img = imgs[i];
            a.pitch = pitches[i];
            a.H = Hs[i];
            a.W = Ws[i];
            a.thr = g_emu_thr;
            a.vec_in = ((uintptr_t)imgs[i] % 16 == 0) && (pitches[i] % 16 == 0);
            a.labels = labels[i];
            a.vec_out = ((uintptr_t)labels[i] % 16 == 0) && (Ws[i] % 4 == 0);
            a.K = Ks + i;
            a.status = status;
            a.gsync = nullptr;
            char *b = (char *)ws[i].data();
            a.nTX = L[i].nTX;
            a.nTY = L[i].nTY;
            a.bitpack = (uint32_t *)(b + L[i].off_bitpack);
            a.cstart = (uint32_t *)(b + L[i].off_cstart);
            a.runinfo = (uint16_t *)(b + L[i].off_runinfo);
            a.nRunInfo = L[i].nRunInfo;
            a.P = (int *)(b + L[i].off_P);
            a.nseg = (int *)(b + L[i].off_nseg);
            a.cnt = (int *)(b + L[i].off_cnt);
            a.edgeRow = (int *)(b + L[i].off_edgeRow);
            a.edgeCol = (int *)(b + L[i].off_edgeCol);
            a.bsum = (int *)(b + L[i].off_bsum);
            a.nP = L[i].nP;
            a.nSeg = L[i].nSeg;
            tileStart[i + 1] = tileStart[i] + (int64_t)L[i].nTX * L[i].nTY;
            itemStart[i + 1] = itemStart[i] + edge_items<C>(L[i].nTX, L[i].nTY, Hs[i], Ws[i]);
            segStart[i + 1] = segStart[i] + L[i].nSeg;
        }
        Batch B;
        memset(&B, 0, sizeof(B));
        B.n = n;
        B.imgs = descs.data();
        B.tileStart = tileStart.data();
        B.itemStart = itemStart.data();
        B.segStart = segStart.data();
        B.imgBase = imgBase.data();
        B.gsync = (GridSync *)(hdr.data() + 16);
        B.bsum = bsum.data();
        B.status = status;
        struct SL2 {
            SmemL<C> s;
            TileCtx ctx;
        };
        struct SF2 {
            SmemF<C> s;
            TileCtx ctx;
        };
        const int ntiles = (int)tileStart[n];
        run_tiles<SL2>(ntiles, [&](SL2 &sm, int tile, int t) { batch_tile_local_body<C>(B, sm.ctx, sm.s, tile, t); });
        const int64_t need = ((itemStart[n] > segStart[n] ? itemStart[n] : segStart[n]) + GNT - 1) / GNT;
        const int G = (int)std::max<int64_t>(1, std::min<int64_t>(3, need));
        std::vector<ScanBuf> sbs(G);
        std::vector<int> flags(G);
        Sched sch(G, GNT, rng(), [&](int b, int t) { batch_global_body<C>(B, sbs[b], flags[b], b, G, t); });
        g_sched = &sch;
        sch.run();
        g_sched = nullptr;
        run_tiles<SF2>(ntiles, [&](SF2 &sm, int tile, int t) { batch_final_body<C>(B, sm.ctx, sm.s, tile, t); });
    }

    int64_t run(const uint8_t *img, int H, int W, int64_t pitch, int32_t *labels, int32_t *status)
    {
        if (H == 0 || W == 0)
            return 0;
        const Layout L = plan_layout<C>(H, W);
        // header (K, status, grid state) + per-image arrays, poisoned
        std::vector<unsigned char> ws((size_t)L.bytes + 256 + 64);
        memset(ws.data(), 0x7B, ws.size());
        char *hdr = (char *)ws.data();
        char *b = hdr + 256;
        Img a;
        memset(&a, 0, sizeof(a));
        a.img = img;
        a.pitch = pitch;
        a.H = H;
        a.W = W;
        a.thr = g_emu_thr;
        a.vec_in = ((uintptr_t)img % 16 == 0) && (pitch % 16 == 0);
        a.labels = labels;
        a.vec_out = ((uintptr_t)labels % 16 == 0) && (W % 4 == 0);
        a.K = (int *)hdr;
        a.status = status;
        a.gsync = (GridSync *)(hdr + 16);
        a.nTX = L.nTX;
        a.nTY = L.nTY;
        a.bitpack = (uint32_t *)(b + L.off_bitpack);
        a.cstart = (uint32_t *)(b + L.off_cstart);
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
        a.pf_dist = (int)(seed % 4);  // successor-tile prefetch distance (0: none)

        const int ntiles = L.nTX * L.nTY;
        run_tiles<SmemL<C>>(ntiles, [&](SmemL<C> &s, int tile, int t) { tile_local_body<C>(a, s, tile, t); });
        const int64_t work = edge_items<C>(L.nTX, L.nTY, H, W);
        const int64_t need = ((work > L.nSeg ? work : L.nSeg) + GNT - 1) / GNT;
        const int G = (int)std::max<int64_t>(1, std::min<int64_t>(3, need));
        if ((seed & 1) == 0 && L.nSeg <= SMALL_SEG_CAP) {
            // the small-image form: one CTA, the node table in shared memory
            auto sm = std::make_unique<SmallSmem>();
            memset(sm.get(), 0x7F, sizeof(SmallSmem));
            Sched sch(1, GNT, rng(), [&](int, int t) { small_global_body<C>(a, *sm, t); });
            g_sched = &sch;
            sch.run();
            g_sched = nullptr;
        } else if ((seed & 3) == 3) {
            // the half-size global CTAs of the one-CTA-per-SM form
            const int64_t need2 = ((work > L.nSeg ? work : L.nSeg) + GNT / 2 - 1) / (GNT / 2);
            run_global<GNT / 2>(a, (int)std::max<int64_t>(1, std::min<int64_t>(4, need2)));
        } else {
            run_global(a, G);
        }
        run_tiles<SmemF<C>>(ntiles, [&](SmemF<C> &s, int tile, int t) { final_body<C>(a, s, tile, t); });
        return *a.K;
    }
};

// Persistent single-launch path (fused_body): CA and CB are the two tile shapes compiled
// into the kernel; G CTAs of NT threads all run at once.  pick/lo/hi/probe as FusedArgs.
// n == 1 uses the inline single-image descriptor (no descriptor arrays).
template <class CA, class CB> struct EmuFused {
    std::mt19937_64 rng;
    explicit EmuFused(uint64_t s) : rng(s) {}

    template <class C> static void bind(Img &a, const Layout &L, char *b)
    {
        a.nTX = L.nTX;
        a.nTY = L.nTY;
        a.bitpack = (uint32_t *)(b + L.off_bitpack);
        a.cstart = (uint32_t *)(b + L.off_cstart);
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
    }

    void run(int n, const uint8_t *const *imgs, const int32_t *Hs, const int32_t *Ws, const int64_t *pitches,
             int32_t *const *labels, int32_t *Ks, const int32_t *pick, int32_t lo, int32_t hi, int32_t probe,
             int32_t G, int32_t *status)
    {
        std::vector<std::vector<unsigned char>> ws(n);
        std::vector<Img> descs[2];
        std::vector<int64_t> pre[2][3];
        for (int k = 0; k < 2; k++) {
            descs[k].resize(n);
            for (int j = 0; j < 3; j++)
                pre[k][j].assign(n + 1, 0);
        }
        std::vector<int> imgBase(n + 1, 0x7B7B7B7B), bsum(MAX_GLOBAL_CTAS, 0x7B7B7B7B);
        std::vector<unsigned char> hdr(256, 0x7B);
        memset(hdr.data() + 16, 0, sizeof(GridSync));  // the host clears the grid state
        for (int i = 0; i < n; i++) {
            const Layout LA = plan_layout<CA>(Hs[i], Ws[i]), LB = plan_layout<CB>(Hs[i], Ws[i]);
            ws[i].assign((size_t)std::max(LA.bytes, LB.bytes) + 64, 0x7B);
            for (int k = 0; k < 2; k++) {
                Img &a = descs[k][i];
                memset(&a, 0, sizeof(a));
                a.img = imgs[i];
                a.pitch = pitches[i];
                a.H = Hs[i];
                a.W = Ws[i];
                a.thr = g_emu_thr;
                a.vec_in = ((uintptr_t)imgs[i] % 16 == 0) && (pitches[i] % 16 == 0);
                a.labels = labels[i];
                a.vec_out = ((uintptr_t)labels[i] % 16 == 0) && (Ws[i] % 4 == 0);
                a.K = Ks + i;
                a.status = status;
                const Layout &L = k ? LB : LA;
                if (k)
                    bind<CB>(a, L, (char *)ws[i].data());
                else
                    bind<CA>(a, L, (char *)ws[i].data());
                pre[k][0][i + 1] = pre[k][0][i] + (int64_t)L.nTX * L.nTY;
                pre[k][1][i + 1] = pre[k][1][i] + (k ? edge_items<CB>(L.nTX, L.nTY, Hs[i], Ws[i])
                                                         : edge_items<CA>(L.nTX, L.nTY, Hs[i], Ws[i]));
                pre[k][2][i + 1] = pre[k][2][i] + L.nSeg;
            }
        }
        FusedArgs f;
        memset(&f, 0, sizeof(f));
        for (int k = 0; k < 2; k++) {
            Batch &B = f.set[k];
            B.n = n;
            B.imgs = descs[k].data();
            B.tileStart = pre[k][0].data();
            B.itemStart = pre[k][1].data();
            B.segStart = pre[k][2].data();
            B.imgBase = imgBase.data();
            B.gsync = (GridSync *)(hdr.data() + 16);
            B.bsum = bsum.data();
            B.status = status;
            if (n == 1) {
                B.inl = 1;
                B.one = descs[k][0];
                B.one_tiles = pre[k][0][1];
                B.one_items = pre[k][1][1];
                B.one_segs = pre[k][2][1];
                B.imgs = nullptr;
                B.tileStart = B.itemStart = B.segStart = nullptr;
            }
        }
        for (int c = 0; c < 3; c++)
            f.pick[c] = pick[c];
        f.dens_lo = lo;
        f.dens_hi = hi;
        f.probe_samples = probe;
        std::vector<std::unique_ptr<FusedSmem<CA, CB>>> sm(G);
        for (auto &p : sm) {
            p.reset(new FusedSmem<CA, CB>);
            memset(p.get(), 0x7F, sizeof(FusedSmem<CA, CB>));
        }
        Sched sch(G, CA::NT, rng(), [&](int b, int t) { fused_body<CA, CB>(f, *sm[b], b, G, t); });
        g_sched = &sch;
        sch.run();
        g_sched = nullptr;
    }
};

}  // namespace

extern "C" {

// the persistent single-launch path on n images (H, W > 0).  pair 0: 8x64 and 4x64 tiles of
// 64 threads (8-connectivity), pair 1: 8x64 alone, pair 2: 4x32 alone under 4-connectivity,
// pair 3: 4x32 alone, multi-class under 8-connectivity.
void emu_label_fused(int32_t n, const uint8_t *const *imgs, const int32_t *H, const int32_t *W, const int64_t *pitch,
                     int32_t *const *labels, int32_t *K, uint64_t seed, int32_t pair, const int32_t *pick,
                     int32_t lo, int32_t hi, int32_t probe, int32_t G, int32_t *status)
{
    *status = 0;
    switch (pair) {
    case 0:
        EmuFused<Cfg<8, 64, 64>, Cfg<4, 64, 64>>(seed).run(n, imgs, H, W, pitch, labels, K, pick, lo, hi, probe, G,
                                                          status);
        break;
    case 1:
        EmuFused<Cfg<8, 64, 64>, Cfg<8, 64, 64>>(seed).run(n, imgs, H, W, pitch, labels, K, pick, lo, hi, probe, G,
                                                          status);
        break;
    case 2:
        EmuFused<Cfg<4, 32, 32, 4>, Cfg<4, 32, 32, 4>>(seed).run(n, imgs, H, W, pitch, labels, K, pick, lo, hi,
                                                                probe, G, status);
        break;
    default:
        EmuFused<Cfg<4, 32, 32, 8, true>, Cfg<4, 32, 32, 8, true>>(seed).run(n, imgs, H, W, pitch, labels, K, pick,
                                                                            lo, hi, probe, G, status);
        break;
    }
}


// threshold of the object test (object = byte > thr) for the following emu_label calls
void emu_set_threshold(int32_t thr) { g_emu_thr = thr; }

// the 4-byte equality test of the multi-class load phase
uint32_t emu_eq_nibble(uint32_t a, uint32_t b) { return ccl::eq_nibble(a, b); }

// the 16-byte object test of the load phase, for an exhaustive check of its arithmetic
uint32_t emu_gt_mask16(const uint8_t *src, int32_t thr)
{
    return ccl::gt_mask16(src, (uint32_t)(255 - thr) * 0x01010101u);
}

// shapes, 8-connectivity: 0 = 64x256 tiles (256 threads); 1 = 4x32 (32); 2 = 8x64 (64);
// 3 = 128x256 (256); 4 = 64x512 (256).  4-connectivity: 5 = 32x256 (256); 6 = 4x32 (32);
// 7 = 8x64 (64); 8 = 2x32 (32).  Multi-class, 8: 9 = 4x32, 10 = 8x64, 11 = 32x256;
// multi-class, 4: 12 = 4x32, 13 = 32x256.  8-connectivity, other tile shapes of the
// tile-shape sweep: 14 = 32x256 (256), 15 = 64x128 (256); 16 = 64x512 (512), the big tiles
int64_t emu_label(const uint8_t *img, int32_t H, int32_t W, int64_t pitch, int32_t *labels, uint64_t seed,
                  int32_t shape, int32_t *status)
{
    *status = 0;
    switch (shape) {
    case 0: return Emu<Cfg<64, 256, 256>>(seed).run(img, H, W, pitch, labels, status);
    case 1: return Emu<Cfg<4, 32, 32>>(seed).run(img, H, W, pitch, labels, status);
    case 2: return Emu<Cfg<8, 64, 64>>(seed).run(img, H, W, pitch, labels, status);
    case 3: return Emu<Cfg<128, 256, 256>>(seed).run(img, H, W, pitch, labels, status);
    case 4: return Emu<Cfg<64, 512, 256>>(seed).run(img, H, W, pitch, labels, status);
    case 5: return Emu<Cfg<32, 256, 256, 4>>(seed).run(img, H, W, pitch, labels, status);
    case 6: return Emu<Cfg<4, 32, 32, 4>>(seed).run(img, H, W, pitch, labels, status);
    case 7: return Emu<Cfg<8, 64, 64, 4>>(seed).run(img, H, W, pitch, labels, status);
    case 8: return Emu<Cfg<2, 32, 32, 4>>(seed).run(img, H, W, pitch, labels, status);
    case 9: return Emu<Cfg<4, 32, 32, 8, true>>(seed).run(img, H, W, pitch, labels, status);
    case 10: return Emu<Cfg<8, 64, 64, 8, true>>(seed).run(img, H, W, pitch, labels, status);
    case 11: return Emu<Cfg<32, 256, 256, 8, true>>(seed).run(img, H, W, pitch, labels, status);
    case 12: return Emu<Cfg<4, 32, 32, 4, true>>(seed).run(img, H, W, pitch, labels, status);
    case 14: return Emu<Cfg<32, 256, 256>>(seed).run(img, H, W, pitch, labels, status);
    case 15: return Emu<Cfg<64, 128, 256>>(seed).run(img, H, W, pitch, labels, status);
    case 16: return Emu<Cfg<64, 512, 512>>(seed).run(img, H, W, pitch, labels, status);
    default: return Emu<Cfg<32, 256, 256, 4, true>>(seed).run(img, H, W, pitch, labels, status);
    }
}

// the batched path; every image must have H, W > 0
void emu_label_batch(int32_t n, const uint8_t *const *imgs, const int32_t *H, const int32_t *W, const int64_t *pitch,
                     int32_t *const *labels, int32_t *K, uint64_t seed, int32_t shape, int32_t *status)
{
    *status = 0;
    switch (shape) {
    case 0: Emu<Cfg<64, 256, 256>>(seed).run_batch(n, imgs, H, W, pitch, labels, K, status); break;
    case 1: Emu<Cfg<4, 32, 32>>(seed).run_batch(n, imgs, H, W, pitch, labels, K, status); break;
    case 2: Emu<Cfg<8, 64, 64>>(seed).run_batch(n, imgs, H, W, pitch, labels, K, status); break;
    case 6: Emu<Cfg<4, 32, 32, 4>>(seed).run_batch(n, imgs, H, W, pitch, labels, K, status); break;
    case 9: Emu<Cfg<4, 32, 32, 8, true>>(seed).run_batch(n, imgs, H, W, pitch, labels, K, status); break;
    case 12: Emu<Cfg<4, 32, 32, 4, true>>(seed).run_batch(n, imgs, H, W, pitch, labels, K, status); break;
    case 15: Emu<Cfg<64, 128, 256>>(seed).run_batch(n, imgs, H, W, pitch, labels, K, status); break;
    default: Emu<Cfg<8, 64, 64, 4>>(seed).run_batch(n, imgs, H, W, pitch, labels, K, status); break;
    }
}

}  // extern "C"
