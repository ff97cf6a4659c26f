// C ABI of the library (declared in include/logan.h): context, options,
// workspace layout, and the batch pipeline
//   [pack] -> validate -> split -> bin -> extension levels -> ring -> combine
// launched asynchronously on the caller's stream, optionally captured into a
// CUDA graph per batch shape and replayed.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ctx_ext.h"
#include "internal.h"
#include "../../include/logan.h"

using namespace logan;

namespace {

constexpr size_t kAlign = 256;
constexpr int kEvSets = 32;        // timed calls whose events are kept
// Launch units: the window levels (0 .. kNumLevels-1), then the latency
// forms of levels 0 .. kTwinLevels-1 (unit kNumLevels + k).
constexpr int kUnits = kNumLevels + kTwinLevels;
inline int unit_queue(int u) { return u < kNumLevels ? u : twin_queue(u - kNumLevels); }
inline int unit_level(int u) { return u < kNumLevels ? u : u - kNumLevels; }

// per timed call: phase-1 start/end and phase-2 start/end of every unit,
// then pipeline start, fallback start, fallback end, pipeline end
constexpr int EV_P1S = 0, EV_P1E = kUnits, EV_P2S = 2 * kUnits, EV_P2E = 3 * kUnits;
constexpr int EV_START = 4 * kUnits, EV_RING_S = EV_START + 1, EV_RING_E = EV_START + 2,
              EV_END = EV_START + 3;
constexpr int kEvPerSet = 4 * kUnits + 4;

// Streams on which the start queues of one caller stream run concurrently.
struct AuxSet {
    cudaStream_t main = nullptr;
    cudaStream_t st[kUnits] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kUnits] = {};
};
inline size_t up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct GraphEntry {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    uint64_t last_use = 0;
};

}  // namespace

struct logan_ctx {
    int device = 0;
    int num_sms = 0;
    int64_t opt_graphs = 0;
    int64_t opt_timing = 0;
    int64_t force_level = -1;
    int64_t max_level = kNumLevels - 1;
    int64_t ring_log2 = 16;
    int64_t plain_level = 1;
    int64_t mig_mb = 64;  // migration records per level, MiB (0: restart on overflow)
    LevelTable table{};
    int blocks_per_sm[kNumLevels] = {};
    int twin_blocks_per_sm[kTwinLevels] = {};
    int affine_blocks_per_sm[4] = {};
    int affine16_blocks_per_sm[4] = {};
    uint32_t affine_packed_last = 0u;  // bit l: affine level l ran packed in the last call
    uint32_t matrix_packed_last = 0u;  // bit l: matrix window l ran packed in the last call
    // LOGAN_OPT_LONG_ITEM: m + n from which items of levels < kTwinLevels
    // take the latency form; -1 never, -2 automatic
    int64_t long_item = -2;
    // LOGAN_OPT_PACKED16: 1 = run a level in its packed 16-bit form when the
    // call's scoring and X provably fit (see packed16_levels), 0 = never
    int64_t packed16 = 1;
    int packed_blocks_per_sm[kNumLevels] = {};
    int8_t next_level[kNumLevels] = {};
    // timing: the events of the last kEvSets timed calls (ring)
    cudaEvent_t evs[kEvSets][kEvPerSet] = {};
    cudaEvent_t* ev = evs[0];      // set of the call in progress / last call
    uint64_t timed_calls = 0;
    struct CallInfo {
        int first_level = 0;
        int max_level = 0;
        uint32_t launches = 0;
        uint32_t p1_levels = 0;  // bit u: phase-1 events of launch unit u recorded
        uint32_t p2_levels = 0;
        bool plain = false;
        uint32_t packed = 0;     // bit l: level l ran in its packed 16-bit form
    } calls[kEvSets];
    // the level counters of each timed call, copied back at its end
    Counters* hcounters = nullptr;  // pinned, kEvSets entries
    int64_t concurrent = 1;  // run the start levels of a batch concurrently
    std::vector<AuxSet> aux;
    bool timing_pending = false;
    uint32_t launches_last = 0;
    // graph cache
    std::vector<GraphEntry> graphs;
    uint64_t use_clock = 0;
    // the last timed alignment-path call
    TracebackTiming tb_timing;
    // scratch of the overlap and alignment-path calls (created on first use)
    cudaMemPool_t scratch_pool = nullptr;
};


namespace {

struct Layout {
    size_t wordsA = 0, wordsB = 0, badA = 0, badB = 0, items = 0, info = 0, ext = 0, queues = 0,
           counters = 0, hist = 0, ring = 0, mig_slot = 0, total = 0;
    size_t mig_pool[kNumLevels] = {};
    uint32_t mig_cap[kNumLevels] = {};
    bool same = false;
    uint32_t ring_slots = 0;
    uint32_t ring_cap = 0;
};

bool same_pool(const logan_seqs_t* a, const logan_seqs_t* b) {
    return a->bases == b->bases && a->offsets == b->offsets && a->lengths == b->lengths &&
           a->count == b->count && a->packed2bit == b->packed2bit && a->pool_bases == b->pool_bases;
}

size_t words_bytes(const logan_seqs_t* s) {
    return s->packed2bit ? 0 : ((s->pool_bases + 15) / 16 + 1) * sizeof(uint32_t);
}

Layout make_layout(const logan_ctx* c, const logan_seqs_t* A, const logan_seqs_t* B, uint32_t n) {
    Layout L;
    L.same = same_pool(A, B);
    const size_t items = size_t(2) * n;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += up(bytes);
        return at;
    };
    L.wordsA = take(words_bytes(A));
    L.wordsB = take(L.same ? 0 : words_bytes(B));
    L.badA = take(A->count);
    L.badB = take(L.same ? 0 : B->count);
    L.items = take(items * sizeof(Item));
    L.info = take(size_t(n) * sizeof(PairInfo));
    L.ext = take(items * sizeof(ExtRes));
    L.queues = take(size_t(kQueues) * items * sizeof(uint32_t));
    L.counters = take(sizeof(Counters));
    L.hist = take(sizeof(uint32_t) * kQueues * kBuckets);
    L.ring_cap = 1u << c->ring_log2;
    L.ring_slots = uint32_t(std::max<size_t>(1, std::min<size_t>(size_t(c->num_sms), items)));
    // six arrays of ring_cap cells per slot: the linear ring uses three, the
    // affine continuation (H on three anti-diagonals, E, F on two) all six
    L.ring = take(size_t(L.ring_slots) * 6 * L.ring_cap * sizeof(int32_t));
    L.mig_slot = take(items * sizeof(int32_t));
    for (int l = 0; l < kNumLevels; ++l) {
        const size_t rec = size_t(mig_stride(l)) * sizeof(int32_t);
        const size_t budget = size_t(c->mig_mb) << 20;
        L.mig_cap[l] = uint32_t(std::min<size_t>({items, budget / rec, size_t(1) << 24}));
        L.mig_pool[l] = take(size_t(L.mig_cap[l]) * rec);
    }
    L.total = off;
    return L;
}

}  // namespace

TracebackTiming* logan::ctx_traceback_timing(logan_ctx_t* c) { return &c->tb_timing; }

void logan::ctx_set_matrix_packed(logan_ctx_t* c, uint32_t levels) { c->matrix_packed_last = levels; }

cudaMemPool_t logan::ctx_scratch_pool(logan_ctx_t* c) {
    if (!c->scratch_pool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = c->device;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        // keep freed scratch mapped between calls: re-mapping gigabytes on
        // every call cost more than the seeding kernels themselves
        uint64_t keep = ~uint64_t(0);
        if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return nullptr;
        }
        c->scratch_pool = p;
    }
    return c->scratch_pool;
}

void logan::extension_views(const logan_ctx_t* c, const logan_seqs_t* A, const logan_seqs_t* B,
                            uint32_t n_pairs, const void* ws, ExtensionViews* v) {
    const Layout L = make_layout(c, A, B, n_pairs);
    const char* w = static_cast<const char*>(ws);
    v->wa = A->packed2bit ? static_cast<const uint32_t*>(A->bases)
                          : reinterpret_cast<const uint32_t*>(w + L.wordsA);
    v->wb = L.same ? v->wa
                   : B->packed2bit ? static_cast<const uint32_t*>(B->bases)
                                   : reinterpret_cast<const uint32_t*>(w + L.wordsB);
    v->items = reinterpret_cast<const Item*>(w + L.items);
    v->ext = reinterpret_cast<const ExtRes*>(w + L.ext);
    v->info = reinterpret_cast<const PairInfo*>(w + L.info);
    v->launches = c->launches_last;
}

namespace {

bool params_ok(int32_t match, int32_t mismatch, int32_t gap, int32_t X) {
    auto a = [](int32_t v) { return v < 0 ? -int64_t(v) : int64_t(v); };
    return a(match) <= kMaxParam && a(mismatch) <= kMaxParam && a(gap) <= kMaxParam && gap <= 0 &&
           mismatch <= match && X >= 0 && X <= kMaxX;
}

bool pool_ok(const logan_seqs_t* s) {
    if (!s || s->packed2bit > 1) return false;
    if (s->count == 0) return true;
    return s->bases && s->offsets && s->lengths;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

void default_table(LevelTable& t) {
    // X class -> first window level.  Band width is about 0.8 X on related
    // reads (X=50: <= 59 rows, X=100: <= 100, X=500: <= 444); a level holds
    // bands up to window - rows-per-lane - 1.
    const int8_t lv[kXClasses] = {0, 1, 2, 2, 3, 4, 6, 7};
    for (int i = 0; i < kXClasses; ++i) t.lv[i] = lv[i];
    t.max_level = kNumLevels - 1;
}

int launch_unit(logan_ctx* c, int u, const KernelArgs& ka, int phase, cudaStream_t s,
                uint32_t packed) {
    cudaError_t e;
    if (u < kNumLevels && ((packed >> u) & 1u)) {
        const int grid = c->num_sms * std::max(1, c->packed_blocks_per_sm[u]);
        e = launch_packed_level_persistent(u, ka, grid, phase, s);
    } else if (u >= kNumLevels) {
        const int l = u - kNumLevels;
        const int grid = c->num_sms * std::max(1, c->twin_blocks_per_sm[l]);
        e = launch_twin_persistent(l, ka, grid, phase, s);
    } else {
        const int grid = c->num_sms * std::max(1, c->blocks_per_sm[u]);
        e = u < kWarpLevels ? launch_warp_level_persistent(u, ka, grid, phase, s)
                            : launch_cta_level(u, ka, grid, phase, s);
    }
    return e == cudaSuccess ? LOGAN_OK : LOGAN_ECUDA;
}

// threshold of m + n for the latency forms in a batch of n_items items
uint32_t long_item_min(const logan_ctx* c, uint32_t n_items) {
    if (c->long_item == -1) return 0xffffffffu;
    if (c->long_item >= 0) return uint32_t(std::min<int64_t>(c->long_item, 0xfffffffe));
    // automatic: a batch that cannot fill the GPU's warps runs every item in
    // latency form; otherwise items of 64K bases and more do
    return n_items <= uint32_t(c->num_sms) * 32u ? 0u : 65536u;
}

// The auxiliary streams of caller stream `s` (created on first use).
AuxSet* aux_for(logan_ctx* c, cudaStream_t s) {
    for (auto& a : c->aux)
        if (a.main == s) return &a;
    AuxSet a;
    a.main = s;
    bool ok = cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int l = 0; ok && l < kUnits; ++l) {
        ok = cudaStreamCreateWithFlags(&a.st[l], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&a.join[l], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        for (int l = 0; l < kUnits; ++l) {
            if (a.st[l]) cudaStreamDestroy(a.st[l]);
            if (a.join[l]) cudaEventDestroy(a.join[l]);
        }
        if (a.fork) cudaEventDestroy(a.fork);
        return nullptr;
    }
    c->aux.push_back(a);
    return &c->aux.back();
}

// Levels that run in their packed 16-bit form in this call: those with a
// packed kernel, when
//   128 * (Xmax + 2*max(match,0) + |gap| + 2) + 31 <= 32767  and
//   128 * (|mismatch| + |gap| + 2*max(match,0) + 2) <= 16383,
// Xmax the largest X that can reach the level: the scalar X when there is
// no per-pair X and no forced start level, else the upper bound of every X
// class whose start level is at or below it (items only move to wider
// levels).  These bounds keep every 16-bit half inside [0, 65536) through
// the kernel's additions (xdrop_group16.cu).
uint32_t packed16_levels(const logan_ctx* c, Scoring sc, int32_t X, const int32_t* Xs,
                         const LevelTable& tab, int64_t force) {
    if (!c->packed16) return 0u;
    static const int64_t upper[kXClasses] = {15, 35, 75, 150, 300, 700, 2000, int64_t(1) << 29};
    const int64_t mp = std::max<int64_t>(sc.match, 0);
    const int64_t ag = -int64_t(sc.gap), am = sc.mismatch < 0 ? -int64_t(sc.mismatch) : sc.mismatch;
    uint32_t mask = 0u;
    for (int l = 0; l < kNumLevels; ++l) {
        if (!packed_level(l) || l > tab.max_level) continue;
        int64_t xmax = 0;
        if (!Xs && force < 0) {
            xmax = X;
        } else if (force >= 0) {
            xmax = force <= l ? (Xs ? upper[kXClasses - 1] : X) : 0;
        } else {
            for (int k = 0; k < kXClasses; ++k)
                if (tab.lv[k] <= l) xmax = std::max(xmax, upper[k]);
        }
        constexpr int64_t S = 128;  // score scale of the packed keys
        if (S * (xmax + 2 * mp + ag + 2) + 31 <= 32767 && S * (am + ag + 2 * mp + 2) <= 16383)
            mask |= 1u << l;
    }
    return mask;
}

// Affine levels that run in their packed 16-bit form in this call: those
// with a packed kernel, when
//   128 * (Xmax + 2*max(match,0) + |go| + |ge| + 2) + 31 <= 32767  and
//   128 * (|mismatch| + |go| + 2*|ge| + 2*max(match,0) + 2) <= 16383,
// Xmax the scalar X, or with per-pair X the upper bound of every X class
// whose start level is at or below the level.  These bounds keep every
// 16-bit half inside [0, 65536) through the kernel's additions
// (xdrop_affine16.cu).
uint32_t affine16_levels(const logan_ctx* c, Scoring sc, int go, int ge, int32_t X,
                         const int32_t* Xs, const LevelTable& tab) {
    if (!c->packed16) return 0u;
    static const int64_t upper[kXClasses] = {15, 35, 75, 150, 300, 700, 2000, int64_t(1) << 29};
    const int64_t mp = std::max<int64_t>(sc.match, 0);
    const int64_t am = sc.mismatch < 0 ? -int64_t(sc.mismatch) : sc.mismatch;
    const int64_t ao = -int64_t(go), ae = -int64_t(ge);
    uint32_t mask = 0u;
    for (int l = 0; l < affine_levels(); ++l) {
        if (!affine16_level(l)) continue;
        int64_t xmax = 0;
        if (!Xs) {
            xmax = X;
        } else {
            for (int k = 0; k < kXClasses; ++k)
                if (tab.lv[k] <= l) xmax = std::max(xmax, upper[k]);
        }
        constexpr int64_t S = 128;  // score scale of the packed keys
        if (S * (xmax + 2 * mp + ao + ae + 2) + 31 <= 32767 &&
            S * (am + ao + 2 * ae + 2 * mp + 2) <= 16383)
            mask |= 1u << l;
    }
    return mask;
}

// The whole pipeline on `s` (no synchronisation).  plain != 0: one-launch
// form at c->plain_level, in input order.
// aff != nullptr: affine gaps (gap_open, gap_extend), through the affine
// window levels instead of the linear ones.
struct AffineGaps {
    int32_t open, extend;
};

int run_pipeline(logan_ctx* c, const logan_seqs_t* A, const logan_seqs_t* B,
                 const logan_seed_t* seeds, uint32_t n_pairs, Scoring sc, int32_t X,
                 const int32_t* Xs, char* ws, const Layout& L, logan_result_t* out,
                 cudaStream_t s, int plain, bool timing, const AffineGaps* aff = nullptr) {
    PoolDev pa = {A->bases, A->offsets, A->lengths, A->count, A->packed2bit, A->pool_bases,
                  A->packed2bit ? static_cast<const uint32_t*>(A->bases)
                                : reinterpret_cast<const uint32_t*>(ws + L.wordsA),
                  reinterpret_cast<uint8_t*>(ws + L.badA)};
    PoolDev pb = pa;
    if (!L.same) {
        pb = {B->bases, B->offsets, B->lengths, B->count, B->packed2bit, B->pool_bases,
              B->packed2bit ? static_cast<const uint32_t*>(B->bases)
                            : reinterpret_cast<const uint32_t*>(ws + L.wordsB),
              reinterpret_cast<uint8_t*>(ws + L.badB)};
    }
    cudaError_t e = cudaSuccess;
    uint32_t launches = 0;
    if (timing) e = cudaEventRecord(c->ev[EV_START], s);
    if (e == cudaSuccess && !A->packed2bit && A->pool_bases) {
        e = launch_pack(pa, reinterpret_cast<uint32_t*>(ws + L.wordsA), s);
        ++launches;
    }
    if (e == cudaSuccess) e = launch_validate(pa, s);
    launches += A->count ? 1 : 0;
    if (!L.same) {
        if (e == cudaSuccess && !B->packed2bit && B->pool_bases) {
            e = launch_pack(pb, reinterpret_cast<uint32_t*>(ws + L.wordsB), s);
            ++launches;
        }
        if (e == cudaSuccess) e = launch_validate(pb, s);
        launches += B->count ? 1 : 0;
    }
    Item* items = reinterpret_cast<Item*>(ws + L.items);
    PairInfo* info = reinterpret_cast<PairInfo*>(ws + L.info);
    ExtRes* ext = reinterpret_cast<ExtRes*>(ws + L.ext);
    uint32_t* queues = reinterpret_cast<uint32_t*>(ws + L.queues);
    Counters* counters = reinterpret_cast<Counters*>(ws + L.counters);
    const uint32_t n_items = 2u * n_pairs;
    if (e == cudaSuccess)
        e = launch_split(pa, pb, seeds, n_pairs, sc, X, Xs, items, info, ext,
                         reinterpret_cast<int32_t*>(ws + L.mig_slot), s);
    ++launches;
    const int maxl = aff ? kNumLevels - 1 : int(c->max_level);
    LevelTable tab = c->table;
    tab.max_level = maxl;
    tab.long_min = long_item_min(c, 2u * n_pairs);
    if (aff) {
        // affine windows 64 / 128 / 256 / 512 rows by X class, longest first;
        // X too large for the affine keys goes to queue kWarpLevels and is
        // rejected
        const int8_t alv[kXClasses] = {0, 0, 1, 1, 2, 3, 3, 3};
        for (int i = 0; i < kXClasses; ++i) tab.lv[i] = alv[i];
        tab.long_min = 0xffffffffu;
    }
    int first = 0;
    if (e == cudaSuccess) {
        if (plain) {
            first = int(std::min<int64_t>(c->plain_level, maxl));
            e = launch_reset_counters(counters, n_items, first, s);
            ++launches;
        } else {
            const int force = (!aff && c->force_level >= 0)
                                  ? int(std::min<int64_t>(c->force_level, maxl))
                                  : -1;
            e = launch_bin(items, n_items, tab, force, reinterpret_cast<uint32_t*>(ws + L.hist), queues,
                           n_items, counters, s);
            launches += 3;
        }
    }
    if (e != cudaSuccess) return LOGAN_ECUDA;
    KernelArgs ka;
    ka.wa = pa.words;
    ka.wb = pb.words;
    ka.items = items;
    ka.ext = ext;
    ka.queues = queues;
    ka.counters = counters;
    ka.ring = reinterpret_cast<int32_t*>(ws + L.ring);
    ka.qcap = n_items;
    ka.n_items = n_items;
    ka.ring_cap = L.ring_cap;
    ka.n_ring_slots = L.ring_slots;
    ka.max_level = uint32_t(maxl);
    ka.sc = sc;
    ka.one = 1;
    for (int k = 0; k < 16; ++k) ka.pw[k] = 1u << (31 - 2 * k);
    for (int k = 0; k < 16; ++k) ka.pw16[k] = 1u << (15 - k);
    for (int l = 0; l < kNumLevels; ++l) {
        ka.next_level[l] = c->next_level[l];
        ka.mig_cap[l] = L.mig_cap[l];
        ka.mig_pool[l] = L.mig_cap[l] ? reinterpret_cast<int32_t*>(ws + L.mig_pool[l]) : nullptr;
    }
    ka.mig_slot = reinterpret_cast<int32_t*>(ws + L.mig_slot);
    const int64_t forced = c->force_level >= 0 ? std::min<int64_t>(c->force_level, maxl) : -1;
    const uint32_t packed = (aff || plain) ? 0u : packed16_levels(c, sc, X, Xs, tab, forced);
    if (aff) {
        // affine levels, narrowest first (each receives the bands that
        // outgrew the previous one), then the rejected items, then combine
        const uint32_t apacked = affine16_levels(c, sc, aff->open, aff->extend, X, Xs, tab);
        for (int l = 0; l < affine_levels(); ++l) {
            cudaError_t le;
            if ((apacked >> l) & 1u) {
                const int grid = c->num_sms * std::max(1, c->affine16_blocks_per_sm[l]);
                le = launch_affine16_level(l, ka, aff->open, aff->extend, affine_levels(), grid, s);
            } else {
                const int grid = c->num_sms * std::max(1, c->affine_blocks_per_sm[l]);
                le = launch_affine_level(l, ka, aff->open, aff->extend, grid, s);
            }
            if (le != cudaSuccess) return LOGAN_ECUDA;
            ++launches;
        }
        c->affine_packed_last = apacked;
        if (launch_affine_ring(ka, kWarpLevels, aff->open, aff->extend, int(L.ring_slots),
                               s) != cudaSuccess ||
            launch_combine(seeds, info, ext, n_pairs, out, s) != cudaSuccess)
            return LOGAN_ECUDA;
        c->launches_last = launches + 2;
        return LOGAN_OK;
    }
    // With one X for the whole batch the host knows every item's start queue
    // (the binning's rule): only those launch in phase 1, and phase 2 starts
    // above that level (a level only receives items from narrower ones).
    uint32_t start_units = ~0u;
    int first_escalated = plain ? first + 1 : 0;
    if (!plain && !Xs) {
        const int64_t forced_start = c->force_level >= 0 ? c->force_level : -1;
        int l = forced_start >= 0 ? int(forced_start) : int(tab.lv[x_class(X)]);
        if (X > kGroupMaxX && l < kWarpLevels) l = kWarpLevels;
        l = std::min(l, maxl);
        start_units = 0u;
        const bool twin_form = l < kTwinLevels;
        if (twin_form && tab.long_min != 0xffffffffu) start_units |= 1u << (kNumLevels + l);
        if (!(twin_form && tab.long_min == 0u)) start_units |= 1u << l;
        first_escalated = l + 1;
    }
    uint32_t p1_levels = 0, p2_levels = 0;
    cudaEvent_t* ev = c->ev;
    auto rec = [&](int idx, cudaStream_t st) {
        return !timing || cudaEventRecord(ev[idx], st) == cudaSuccess;
    };
    if (plain) {
        // phase 1: the one-launch form at `first`, in input order
        if (!rec(EV_P1S + first, s)) return LOGAN_ECUDA;
        e = first < kWarpLevels
                ? launch_warp_level_plain(first, ka, s)
                : launch_cta_level(first, ka, c->num_sms * std::max(1, c->blocks_per_sm[first]),
                                   PHASE_PLAIN, s);
        if (e != cudaSuccess || !rec(EV_P1E + first, s)) return LOGAN_ECUDA;
        p1_levels |= 1u << first;
        ++launches;
    } else {
        // phase 1: every queue's binned items; the queues share no entry, so
        // they run concurrently on their own streams, the latency forms
        // (long items) first
        AuxSet* ax = c->concurrent ? aux_for(c, s) : nullptr;
        if (ax && cudaEventRecord(ax->fork, s) != cudaSuccess) return LOGAN_ECUDA;
        for (int k = 0; k < kUnits; ++k) {
            const int u = k < kTwinLevels ? kNumLevels + k : k - kTwinLevels;
            if (unit_level(u) > maxl || !((start_units >> u) & 1u)) continue;
            cudaStream_t st = ax ? ax->st[u] : s;
            if (ax && cudaStreamWaitEvent(st, ax->fork, 0) != cudaSuccess) return LOGAN_ECUDA;
            if (!rec(EV_P1S + u, st)) return LOGAN_ECUDA;
            if (launch_unit(c, u, ka, PHASE_INITIAL, st, packed) != LOGAN_OK) return LOGAN_ECUDA;
            if (!rec(EV_P1E + u, st)) return LOGAN_ECUDA;
            if (ax && (cudaEventRecord(ax->join[u], st) != cudaSuccess ||
                       cudaStreamWaitEvent(s, ax->join[u], 0) != cudaSuccess))
                return LOGAN_ECUDA;
            p1_levels |= 1u << u;
            ++launches;
        }
    }
    // phase 2: escalated items, narrowest level first (a queue only receives
    // items from narrower levels); a level's latency form after the level
    for (int lvl = first_escalated; lvl <= maxl; ++lvl) {
        for (int u : {lvl, lvl < kTwinLevels && !plain ? kNumLevels + lvl : -1}) {
            if (u < 0) continue;
            if (!rec(EV_P2S + u, s)) return LOGAN_ECUDA;
            if (launch_unit(c, u, ka, PHASE_ESCALATED, s, packed) != LOGAN_OK) return LOGAN_ECUDA;
            if (!rec(EV_P2E + u, s)) return LOGAN_ECUDA;
            p2_levels |= 1u << u;
            ++launches;
        }
    }
    // ring fallback: one resident block per ring slot
    if (!rec(EV_RING_S, s)) return LOGAN_ECUDA;
    if (launch_ring(ka, int(L.ring_slots), s) != cudaSuccess) return LOGAN_ECUDA;
    if (!rec(EV_RING_E, s)) return LOGAN_ECUDA;
    if (launch_combine(seeds, info, ext, n_pairs, out, s) != cudaSuccess) return LOGAN_ECUDA;
    launches += 2;  // ring + combine
    c->launches_last = launches;
    if (timing) {
        if (cudaMemcpyAsync(&c->hcounters[c->timed_calls % kEvSets], counters, sizeof(Counters),
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            !rec(EV_END, s))
            return LOGAN_ECUDA;
        auto& ci = c->calls[c->timed_calls % kEvSets];
        ci.first_level = plain ? first : 0;
        ci.max_level = maxl;
        ci.launches = launches;
        ci.p1_levels = p1_levels;
        ci.p2_levels = p2_levels;
        ci.plain = plain != 0;
        ci.packed = packed;
        c->timed_calls += 1;
        c->timing_pending = true;
    }
    return LOGAN_OK;
}

int extend_common(logan_ctx* c, const logan_seqs_t* A, const logan_seqs_t* B,
                  const logan_seed_t* seeds, uint32_t n_pairs, int32_t match, int32_t mismatch,
                  int32_t gap, int32_t X, const int32_t* Xs, void* ws, size_t ws_bytes,
                  logan_result_t* out, void* stream, int plain) {
    if (!c || !pool_ok(A) || !pool_ok(B)) return LOGAN_EINVAL;
    if (!params_ok(match, mismatch, gap, X)) return LOGAN_EINVAL;
    if (n_pairs > 0x7fffffffu) return LOGAN_EINVAL;
    if (n_pairs == 0) return LOGAN_OK;
    if (!seeds || !out || !ws) return LOGAN_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return LOGAN_EINVAL;
    const Layout L = make_layout(c, A, B, n_pairs);
    if (ws_bytes < L.total) return LOGAN_ENOMEM;
    DeviceGuard g(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Scoring sc = {match, mismatch, gap};
    const bool timing = c->opt_timing != 0;
    if (timing) c->ev = c->evs[c->timed_calls % kEvSets];
    if (!c->opt_graphs || timing || s == nullptr)
        return run_pipeline(c, A, B, seeds, n_pairs, sc, X, Xs, static_cast<char*>(ws), L, out, s,
                            plain, timing);
    // graph path: key = everything the launch sequence depends on
    std::vector<uint64_t> key = {
        uint64_t(plain), uint64_t(n_pairs), uint64_t(uint32_t(match)), uint64_t(uint32_t(mismatch)),
        uint64_t(uint32_t(gap)), uint64_t(uint32_t(X)), uint64_t(uintptr_t(Xs)),
        uint64_t(uintptr_t(seeds)), uint64_t(uintptr_t(out)), uint64_t(uintptr_t(ws)),
        uint64_t(uintptr_t(stream)), uint64_t(c->force_level), uint64_t(c->max_level),
        uint64_t(c->ring_log2), uint64_t(c->plain_level), uint64_t(c->mig_mb),
        uint64_t(c->concurrent), uint64_t(c->long_item), uint64_t(c->packed16)};
    for (const logan_seqs_t* p : {A, B}) {
        key.push_back(uint64_t(uintptr_t(p->bases)));
        key.push_back(uint64_t(uintptr_t(p->offsets)));
        key.push_back(uint64_t(uintptr_t(p->lengths)));
        key.push_back(uint64_t(p->count) | (uint64_t(p->packed2bit) << 32));
        key.push_back(p->pool_bases);
    }
    for (int i = 0; i < kXClasses; ++i) key.push_back(uint64_t(uint8_t(c->table.lv[i])));
    for (int i = 0; i < kNumLevels; ++i) key.push_back(uint64_t(uint8_t(c->next_level[i])));
    GraphEntry* hit = nullptr;
    for (auto& ge : c->graphs)
        if (ge.key == key) hit = &ge;
    if (!hit) {
        // the auxiliary streams are created outside the capture
        if (c->concurrent && !plain && !aux_for(c, s)) return LOGAN_ECUDA;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return LOGAN_ECUDA;
        int rc = run_pipeline(c, A, B, seeds, n_pairs, sc, X, Xs, static_cast<char*>(ws), L, out, s,
                              plain, false);
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (rc || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc ? rc : LOGAN_ECUDA;
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return LOGAN_ECUDA;
        if (c->graphs.size() >= 8) {
            auto oldest = c->graphs.begin();
            for (auto it = c->graphs.begin(); it != c->graphs.end(); ++it)
                if (it->last_use < oldest->last_use) oldest = it;
            cudaGraphExecDestroy(oldest->exec);
            c->graphs.erase(oldest);
        }
        c->graphs.push_back(GraphEntry{key, exec, 0});
        hit = &c->graphs.back();
    }
    hit->last_use = ++c->use_clock;
    return cudaGraphLaunch(hit->exec, s) == cudaSuccess ? LOGAN_OK : LOGAN_ECUDA;
}

int set_table(logan_ctx_t* c, const int8_t* levels, int n) {
    if (!c || !levels || n != kXClasses) return LOGAN_EINVAL;
    for (int i = 0; i < n; ++i)
        if (levels[i] < 0 || levels[i] >= kNumLevels) return LOGAN_EINVAL;
    for (int i = 0; i < n; ++i) c->table.lv[i] = levels[i];
    return LOGAN_OK;
}

int load_table_json(logan_ctx_t* c, const char* path) {
    FILE* f = std::fopen(path, "rb");
    if (!f) return LOGAN_EINVAL;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    const size_t at = text.find("\"levels\"");
    if (at == std::string::npos) return LOGAN_EINVAL;
    size_t p = text.find('[', at);
    if (p == std::string::npos) return LOGAN_EINVAL;
    int8_t lv[kXClasses];
    for (int i = 0; i < kXClasses; ++i) {
        char* end = nullptr;
        const long v = std::strtol(text.c_str() + p + 1, &end, 10);
        if (!end || end == text.c_str() + p + 1) return LOGAN_EINVAL;
        lv[i] = int8_t(v);
        p = size_t(end - text.c_str());
        if (i + 1 < kXClasses) {
            p = text.find(',', p);
            if (p == std::string::npos) return LOGAN_EINVAL;
        }
    }
    int rc = set_table(c, lv, kXClasses);
    // optional unit-form choices of the autotuner
    const size_t pk = text.find("\"packed16\"");
    if (rc == LOGAN_OK && pk != std::string::npos) {
        const size_t colon = text.find(':', pk);
        if (colon == std::string::npos) return LOGAN_EINVAL;
        c->packed16 = std::strtol(text.c_str() + colon + 1, nullptr, 10) ? 1 : 0;
    }
    const size_t li = text.find("\"long_item\"");
    if (rc == LOGAN_OK && li != std::string::npos) {
        const size_t colon = text.find(':', li);
        if (colon == std::string::npos) return LOGAN_EINVAL;
        const long long v = std::strtoll(text.c_str() + colon + 1, nullptr, 10);
        if (v < -2) return LOGAN_EINVAL;
        c->long_item = v;
    }
    return rc;
}

}  // namespace

extern "C" {

const char* logan_version(void) { return "logan-gb300 0.1 (sm_103a)"; }

const char* logan_strerror(int code) {
    switch (code) {
        case LOGAN_OK: return "ok";
        case LOGAN_EINVAL: return "invalid argument or invalid pair input";
        case LOGAN_ENOMEM: return "workspace too small or host allocation failed";
        case LOGAN_EAGAIN: return "request exceeds the free serving budget";
        case LOGAN_ECUDA: return "CUDA runtime call failed";
        case LOGAN_ETIMEOUT: return "bounded wait expired";
        case LOGAN_ECANCELED: return "request cancelled";
        case LOGAN_ERANGE: return "band wider than the fallback window";
        case LOGAN_ENOTFOUND: return "unknown ticket";
        default: return "unknown error";
    }
}

int logan_ctx_create(logan_ctx_t** out, int device, const char* autotune_json) {
    if (!out) return LOGAN_EINVAL;
    *out = nullptr;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev)
        return LOGAN_ECUDA;
    logan_ctx* c = new (std::nothrow) logan_ctx();
    if (!c) return LOGAN_ENOMEM;
    c->device = device;
    DeviceGuard g(device);
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return LOGAN_ECUDA;
    }
    default_table(c->table);
    // escalation: level+1.  With band-state migration a growing band moves
    // through every window size without repeating work (measured on the
    // 100K-pair batch at X = 100: 354 ms, against 374 ms when the 128-row
    // level escalates straight to the 1024-row level)
    for (int l = 0; l < kNumLevels; ++l) c->next_level[l] = int8_t(l + 1);
    for (int l = 0; l < kNumLevels; ++l)
        c->blocks_per_sm[l] = l < kWarpLevels ? warp_level_blocks_per_sm(l) : cta_level_blocks_per_sm(l);
    for (int l = 0; l < kNumLevels; ++l)
        c->packed_blocks_per_sm[l] = packed_level(l) ? packed_level_blocks_per_sm(l) : 0;
    for (int l = 0; l < kTwinLevels; ++l) c->twin_blocks_per_sm[l] = twin_blocks_per_sm(l);
    for (int l = 0; l < affine_levels(); ++l) {
        c->affine_blocks_per_sm[l] = affine_blocks_per_sm(l);
        c->affine16_blocks_per_sm[l] = affine16_level(l) ? affine16_blocks_per_sm(l) : 0;
    }
    for (auto& set : c->evs)
        for (auto& ev : set)
            if (cudaEventCreate(&ev) != cudaSuccess) {
                logan_ctx_destroy(c);
                return LOGAN_ECUDA;
            }
    if (cudaHostAlloc(reinterpret_cast<void**>(&c->hcounters), sizeof(Counters) * kEvSets,
                      cudaHostAllocDefault) != cudaSuccess) {
        logan_ctx_destroy(c);
        return LOGAN_ECUDA;
    }
    if (autotune_json) {
        int rc = load_table_json(c, autotune_json);
        if (rc) {
            logan_ctx_destroy(c);
            return rc;
        }
    }
    *out = c;
    return LOGAN_OK;
}

void logan_ctx_destroy(logan_ctx_t* c) {
    if (!c) return;
    DeviceGuard g(c->device);
    if (c->scratch_pool) cudaMemPoolDestroy(c->scratch_pool);  // (its memory goes back now)
    for (auto& ge : c->graphs)
        if (ge.exec) cudaGraphExecDestroy(ge.exec);
    for (auto& a : c->aux) {
        for (int l = 0; l < kUnits; ++l) {
            if (a.st[l]) {
                cudaStreamSynchronize(a.st[l]);
                cudaStreamDestroy(a.st[l]);
            }
            if (a.join[l]) cudaEventDestroy(a.join[l]);
        }
        if (a.fork) cudaEventDestroy(a.fork);
    }
    for (auto& set : c->evs)
        for (auto& ev : set)
            if (ev) cudaEventDestroy(ev);
    if (c->hcounters) cudaFreeHost(c->hcounters);
    delete c;
}

int logan_workspace_size(const logan_ctx_t* c, const logan_seqs_t* A, const logan_seqs_t* B,
                         uint32_t n_pairs, size_t* bytes) {
    if (!c || !bytes || !pool_ok(A) || !pool_ok(B)) return LOGAN_EINVAL;
    *bytes = make_layout(c, A, B, n_pairs).total;
    return LOGAN_OK;
}

int logan_extend_batch(logan_ctx_t* c, const logan_seqs_t* A, const logan_seqs_t* B,
                       const logan_seed_t* seeds, uint32_t n_pairs, int32_t match, int32_t mismatch,
                       int32_t gap, int32_t X, const int32_t* Xs, void* ws, size_t ws_bytes,
                       logan_result_t* out, void* stream) {
    return extend_common(c, A, B, seeds, n_pairs, match, mismatch, gap, X, Xs, ws, ws_bytes, out,
                         stream, 0);
}

int logan_extend_batch_plain(logan_ctx_t* c, const logan_seqs_t* A, const logan_seqs_t* B,
                             const logan_seed_t* seeds, uint32_t n_pairs, int32_t match,
                             int32_t mismatch, int32_t gap, int32_t X, const int32_t* Xs, void* ws,
                             size_t ws_bytes, logan_result_t* out, void* stream) {
    return extend_common(c, A, B, seeds, n_pairs, match, mismatch, gap, X, Xs, ws, ws_bytes, out,
                         stream, 1);
}

int logan_extend_batch_affine(logan_ctx_t* c, const logan_seqs_t* A, const logan_seqs_t* B,
                              const logan_seed_t* seeds, uint32_t n_pairs, int32_t match,
                              int32_t mismatch, int32_t gap_open, int32_t gap_extend, int32_t X,
                              const int32_t* Xs, void* ws, size_t ws_bytes, logan_result_t* out,
                              void* stream) {
    if (!c || !pool_ok(A) || !pool_ok(B)) return LOGAN_EINVAL;
    // gap_open + gap_extend is the largest single-step gap penalty: the
    // per-pair range check of the split uses it like the linear gap
    if (!params_ok(match, mismatch, gap_extend, X) || gap_open > 0 ||
        gap_open < -kMaxParam)
        return LOGAN_EINVAL;
    if (n_pairs > 0x7fffffffu) return LOGAN_EINVAL;
    if (n_pairs == 0) return LOGAN_OK;
    if (!seeds || !out || !ws) return LOGAN_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return LOGAN_EINVAL;
    const Layout L = make_layout(c, A, B, n_pairs);
    if (ws_bytes < L.total) return LOGAN_ENOMEM;
    DeviceGuard g(c->device);
    const Scoring sc = {match, mismatch, gap_open + gap_extend};
    const AffineGaps aff = {gap_open, gap_extend};
    return run_pipeline(c, A, B, seeds, n_pairs, sc, X, Xs, static_cast<char*>(ws), L, out,
                        static_cast<cudaStream_t>(stream), 0, false, &aff);
}

int logan_set_option(logan_ctx_t* c, int option, int64_t v) {
    if (!c) return LOGAN_EINVAL;
    switch (option) {
        case LOGAN_OPT_GRAPHS: c->opt_graphs = v ? 1 : 0; return LOGAN_OK;
        case LOGAN_OPT_TIMING: c->opt_timing = v ? 1 : 0; return LOGAN_OK;
        case LOGAN_OPT_FORCE_LEVEL:
            if (v < -1 || v >= kNumLevels) return LOGAN_EINVAL;
            c->force_level = v;
            return LOGAN_OK;
        case LOGAN_OPT_MAX_LEVEL:
            if (v < 0 || v >= kNumLevels) return LOGAN_EINVAL;
            c->max_level = v;
            return LOGAN_OK;
        case LOGAN_OPT_RING_CAP:
            if (v < 10 || v > 22) return LOGAN_EINVAL;
            c->ring_log2 = v;
            return LOGAN_OK;
        case LOGAN_OPT_PLAIN_LEVEL:
            if (v < 0 || v >= kNumLevels) return LOGAN_EINVAL;
            c->plain_level = v;
            return LOGAN_OK;
        case LOGAN_OPT_MIGRATION_MB:
            if (v < 0 || v > 4096) return LOGAN_EINVAL;
            c->mig_mb = v;
            return LOGAN_OK;
        case LOGAN_OPT_CONCURRENT: c->concurrent = v ? 1 : 0; return LOGAN_OK;
        case LOGAN_OPT_LONG_ITEM:
            if (v < -2) return LOGAN_EINVAL;
            c->long_item = v;
            return LOGAN_OK;
        case LOGAN_OPT_PACKED16: c->packed16 = v ? 1 : 0; return LOGAN_OK;
        default: return LOGAN_EINVAL;
    }
}

int logan_get_option(const logan_ctx_t* c, int option, int64_t* v) {
    if (!c || !v) return LOGAN_EINVAL;
    switch (option) {
        case LOGAN_OPT_GRAPHS: *v = c->opt_graphs; return LOGAN_OK;
        case LOGAN_OPT_TIMING: *v = c->opt_timing; return LOGAN_OK;
        case LOGAN_OPT_FORCE_LEVEL: *v = c->force_level; return LOGAN_OK;
        case LOGAN_OPT_MAX_LEVEL: *v = c->max_level; return LOGAN_OK;
        case LOGAN_OPT_RING_CAP: *v = c->ring_log2; return LOGAN_OK;
        case LOGAN_OPT_PLAIN_LEVEL: *v = c->plain_level; return LOGAN_OK;
        case LOGAN_OPT_DEVICE: *v = c->device; return LOGAN_OK;
        case LOGAN_OPT_MIGRATION_MB: *v = c->mig_mb; return LOGAN_OK;
        case LOGAN_OPT_CONCURRENT: *v = c->concurrent; return LOGAN_OK;
        case LOGAN_OPT_LONG_ITEM: *v = c->long_item; return LOGAN_OK;
        case LOGAN_OPT_PACKED16: *v = c->packed16; return LOGAN_OK;
        case LOGAN_OPT_AFFINE_PACKED: *v = c->affine_packed_last; return LOGAN_OK;
        case LOGAN_OPT_MATRIX_PACKED: *v = c->matrix_packed_last; return LOGAN_OK;
        default: return LOGAN_EINVAL;
    }
}

int logan_num_levels(void) { return kNumLevels; }

int logan_level_info(int level, int* window_cells, int* threads_per_unit) {
    if (level < 0 || level >= kNumLevels) return LOGAN_EINVAL;
    if (window_cells) *window_cells = level_window(level);
    if (threads_per_unit) *threads_per_unit = level_threads(level);
    return LOGAN_OK;
}

int logan_call_stats(logan_ctx_t* c, int back, logan_stats_t* st) {
    if (!c || !st || back < 0 || back >= kEvSets) return LOGAN_EINVAL;
    if (!c->timing_pending || uint64_t(back) >= c->timed_calls) return LOGAN_EINVAL;
    static_assert(kNumLevels <= LOGAN_MAX_LEVELS, "stats layout");
    DeviceGuard g(c->device);
    const uint64_t call = c->timed_calls - 1 - uint64_t(back);
    cudaEvent_t* ev = c->evs[call % kEvSets];
    const auto& ci = c->calls[call % kEvSets];
    if (cudaEventSynchronize(ev[EV_END]) != cudaSuccess) return LOGAN_ECUDA;
    std::memset(st, 0, sizeof(*st));
    const Counters& h = c->hcounters[call % kEvSets];
    // a launch counts only if it had entries to process: an empty launch's
    // span is mostly its wait for room on the SMs; a latency form's time
    // and items count for its level
    for (int u = 0; u < kUnits; ++u) {
        const int q = unit_queue(u), l = unit_level(u);
        float ms = 0.f;
        if (((ci.p1_levels >> u) & 1u) && (h.started[q] > 0 || ci.plain)) {
            if (cudaEventElapsedTime(&ms, ev[EV_P1S + u], ev[EV_P1E + u]) != cudaSuccess)
                return LOGAN_ECUDA;
            st->level_ms[l] += ms;
        }
        if (((ci.p2_levels >> u) & 1u) && h.tail[q] > h.started[q]) {
            if (cudaEventElapsedTime(&ms, ev[EV_P2S + u], ev[EV_P2E + u]) != cudaSuccess)
                return LOGAN_ECUDA;
            st->level_ms[l] += ms;
        }
    }
    if (cudaEventElapsedTime(&st->level_ms[kNumLevels], ev[EV_RING_S], ev[EV_RING_E]) != cudaSuccess)
        return LOGAN_ECUDA;
    if (cudaEventElapsedTime(&st->total_ms, ev[EV_START], ev[EV_END]) != cudaSuccess)
        return LOGAN_ECUDA;
    for (int l = 0; l <= kNumLevels; ++l) {
        st->items[l] = h.tail[l] + (l < kTwinLevels ? h.tail[twin_queue(l)] : 0u);
        st->cells[l] = h.cells[l];
    }
    st->launches = ci.launches;
    st->packed_levels = ci.packed;
    return LOGAN_OK;
}

int logan_last_stats(logan_ctx_t* c, logan_stats_t* st) { return logan_call_stats(c, 0, st); }

// ---- autotuner: X class -> fastest start level ----

int logan_autotune(logan_ctx_t* c, const logan_seqs_t* A, const logan_seqs_t* B,
                   const logan_seed_t* seeds, uint32_t n_pairs, int32_t match, int32_t mismatch,
                   int32_t gap, int32_t X, const int32_t* Xs, void* ws, size_t ws_bytes,
                   logan_result_t* out, void* stream, int reps, float* ms_table) {
    if (!c || reps < 1 || n_pairs == 0) return LOGAN_EINVAL;
    DeviceGuard g(c->device);
    // which X classes does the sample hold?
    bool present[kXClasses] = {};
    if (Xs) {
        std::vector<int32_t> hx(n_pairs);
        if (cudaMemcpy(hx.data(), Xs, sizeof(int32_t) * n_pairs, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return LOGAN_ECUDA;
        for (int32_t v : hx)
            if (v >= 0 && v <= kMaxX) present[x_class(v)] = true;
    } else {
        present[x_class(X)] = true;
    }
    const int64_t save_packed = c->packed16, save_long = c->long_item;
    const LevelTable save_table = c->table;
    const int maxl = int(c->max_level);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess)
                 ? LOGAN_OK
                 : LOGAN_ECUDA;
    // one configuration, timed as a caller runs it: the context's graph and
    // timing options, an event pair around the whole call on the caller's
    // stream; one untimed call first (it captures the configuration's
    // graph), then the fastest of `reps`
    auto time_call = [&](float* best) {
        float t_min = -1.f;
        for (int r = -1; r < reps && rc == LOGAN_OK; ++r) {
            if (cudaEventRecord(e0, s) != cudaSuccess) rc = LOGAN_ECUDA;
            if (rc == LOGAN_OK)
                rc = extend_common(c, A, B, seeds, n_pairs, match, mismatch, gap, X, Xs, ws,
                                   ws_bytes, out, stream, 0);
            float t = 0.f;
            if (rc == LOGAN_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                                   cudaEventSynchronize(e1) != cudaSuccess ||
                                   cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
                rc = LOGAN_ECUDA;
            if (rc == LOGAN_OK && r >= 0 && (t_min < 0.f || t < t_min)) t_min = t;
        }
        *best = t_min;
    };
    int8_t chosen[kXClasses];
    for (int k = 0; k < kXClasses; ++k) chosen[k] = save_table.lv[k];
    if (ms_table)
        for (int k = 0; k < kXClasses * kNumLevels; ++k) ms_table[k] = -1.f;
    // A candidate replaces the current choice only when it ran at least 3 %
    // faster: step times of a batch vary by a few per cent between calls,
    // and a choice made on that noise can cost far more on the next call.
    constexpr float kGain = 0.97f;
    // the start level of each X class present: one pass of coordinate
    // descent on the whole sample -- every level for one class, the other
    // classes at their current choice
    for (int cls = 0; cls < kXClasses && rc == LOGAN_OK; ++cls) {
        if (!present[cls]) continue;
        float best_ms = 0.f, cur_ms = -1.f;
        int best_level = -1;
        for (int lvl = 0; lvl <= maxl && rc == LOGAN_OK; ++lvl) {
            int8_t trial[kXClasses];
            for (int k = 0; k < kXClasses; ++k) trial[k] = chosen[k];
            trial[cls] = int8_t(lvl);
            rc = set_table(c, trial, kXClasses);
            float t = -1.f;
            if (rc == LOGAN_OK) time_call(&t);
            if (rc != LOGAN_OK) break;
            if (ms_table) ms_table[cls * kNumLevels + lvl] = t;
            if (lvl == chosen[cls]) cur_ms = t;
            if (best_level < 0 || t < best_ms) {
                best_ms = t;
                best_level = lvl;
            }
        }
        if (best_level >= 0 && (cur_ms < 0.f || best_ms < kGain * cur_ms))
            chosen[cls] = int8_t(best_level);
    }
    c->table = save_table;
    if (rc == LOGAN_OK) rc = set_table(c, chosen, kXClasses);
    // the unit forms with the chosen table: packed 16-bit vs 32-bit, crossed
    // with the one-warp rule
    if (rc == LOGAN_OK) {
        const int64_t forms[4][2] = {{1, -2}, {1, -1}, {0, -2}, {0, -1}};
        float best_ms = -1.f, cur_ms = -1.f;
        int best_form = -1;
        for (int f = 0; f < 4 && rc == LOGAN_OK; ++f) {
            c->packed16 = forms[f][0];
            c->long_item = forms[f][1];
            float t = -1.f;
            time_call(&t);
            if (rc != LOGAN_OK) break;
            if (forms[f][0] == save_packed && forms[f][1] == save_long) cur_ms = t;
            if (best_form < 0 || t < best_ms) {
                best_ms = t;
                best_form = f;
            }
        }
        const bool take = best_form >= 0 && (cur_ms < 0.f || best_ms < kGain * cur_ms);
        c->packed16 = take ? forms[best_form][0] : save_packed;
        c->long_item = take ? forms[best_form][1] : save_long;
    } else {
        c->packed16 = save_packed;
        c->long_item = save_long;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

int logan_autotune_save(const logan_ctx_t* c, const char* path) {
    if (!c || !path) return LOGAN_EINVAL;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) return LOGAN_ECUDA;
    FILE* f = std::fopen(path, "wb");
    if (!f) return LOGAN_EINVAL;
    std::fprintf(f, "{\"gpu\": \"%s\", \"sms\": %d, \"x_class_upper\": [15, 35, 75, 150, 300, 700, 2000, 536870912], \"levels\": [",
                 prop.name, prop.multiProcessorCount);
    for (int i = 0; i < kXClasses; ++i) std::fprintf(f, "%s%d", i ? ", " : "", int(c->table.lv[i]));
    std::fprintf(f, "], \"packed16\": %d, \"long_item\": %lld}\n", int(c->packed16),
                 static_cast<long long>(c->long_item));
    return std::fclose(f) == 0 ? LOGAN_OK : LOGAN_EINVAL;
}

// ---- level table (autotune results) ----

int logan_set_level_table(logan_ctx_t* c, const int8_t* levels, int n) {
    return set_table(c, levels, n);
}

int logan_set_escalation(logan_ctx_t* c, const int8_t* next, int n) {
    if (!c || !next || n != kNumLevels) return LOGAN_EINVAL;
    for (int l = 0; l < n; ++l)
        if (next[l] <= l || next[l] > kNumLevels) return LOGAN_EINVAL;
    for (int l = 0; l < n; ++l) c->next_level[l] = next[l];
    return LOGAN_OK;
}

int logan_get_escalation(const logan_ctx_t* c, int8_t* next, int n) {
    if (!c || !next || n != kNumLevels) return LOGAN_EINVAL;
    for (int l = 0; l < n; ++l) next[l] = c->next_level[l];
    return LOGAN_OK;
}

int logan_get_level_table(const logan_ctx_t* c, int8_t* levels, int n) {
    if (!c || !levels || n != kXClasses) return LOGAN_EINVAL;
    for (int i = 0; i < n; ++i) levels[i] = c->table.lv[i];
    return LOGAN_OK;
}

}  // extern "C"
