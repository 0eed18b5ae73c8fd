// Serving loop of include/screen.h.  Three threads per server:
//  - two builders build the tables of uploaded images and rebuild evicted ones
//    from their host copy (each on its own stream), admitting new tables by the
//    table budget: they evict least recently used tables that no ready or
//    running screen pins, and wait for pins to be released when that is not
//    enough;
//  - the screener serves the screens whose tables are resident.  Batched mode
//    (continuous batching): each turn it takes every ready screen, orders them
//    shortest first and enqueues each one's screening kernel and compaction
//    without waiting (small screens on a higher-priority stream), then retires
//    every screen whose own work has completed; plain mode runs one screen at
//    a time and waits for it.  Lists come back in the single-image key format.
// Copies and table builds of the builders overlap with the screener's kernels.
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>

#include <time.h>

#include "runtime.h"

using namespace scr;
using namespace scr_rt;

namespace {

int64_t now_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

enum { kUpload = 0, kScreen = 1, kEvict = 2 };

struct SrvRequest;

struct SrvImage {
    int64_t id = 0;
    const uint8_t *host = nullptr;   // pixels (own copy or borrowed)
    std::vector<uint8_t> own;
    int H = 0, W = 0;
    int64_t pitch = 0;
    // everything below is read and written under the server lock
    scr_tables *t = nullptr;         // resident tables, or null
    uint64_t last_use = 0;           // LRU stamp
    int builds = 0;
    int refs = 0;                    // submitted requests naming the image, not yet completed
    int pins = 0;                    // ready or running screens using the tables
    bool building = false;           // a build job is queued or running
    bool forgotten = false;          // dropped by server_forget; freed once refs == 0 and not building
    std::vector<SrvRequest *> waiting;   // screens waiting for the build
};

struct SrvRequest {
    uint64_t id = 0;
    int kind = kScreen;
    SrvImage *img = nullptr;
    const scr_tmpl *tm = nullptr;
    scr_params p = {};
    std::vector<int32_t> radii;
    uint64_t *list_host = nullptr;
    uint64_t list_cap = 0;
    bool done = false;
    scr_request_result res = {};
};

struct BuildJob {
    SrvImage *img;
    SrvRequest *req;   // the upload or evict request, or null for a rebuild
};

// device or pinned host buffer that only grows
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct scr_server {
    scr_ctx *ctx = nullptr;
    scr_server_config cfg = {};
    std::mutex mu;
    std::condition_variable cv_screen, cv_build, cv_unpin, cv_done;
    std::deque<SrvRequest *> pending;                  // submitted, not yet sorted by the screener
    std::vector<SrvRequest *> ready;                   // screens with pinned resident tables
    std::deque<BuildJob> jobs;                         // builder queue
    std::unordered_map<uint64_t, SrvRequest *> reqs;   // submitted, not yet collected
    std::deque<uint64_t> done_q;                       // completed ids, in completion order
    std::unordered_map<int64_t, SrvImage *> images;
    std::vector<SrvImage *> dropped;                   // forgotten images to free (builder)
    uint64_t next_req = 1;
    int64_t next_image = 1;
    bool stop = false, hold = false, stop_builder = false;
    int jobs_in_flight = 0;
    std::thread screener;
    cudaStream_t st = nullptr;                         // screener stream
    struct Builder {                                   // builders work on different images at once
        std::thread th;
        cudaStream_t st = nullptr;
        DevBuf img;                                    // the image on the device while its tables build
        DevBuf scratch;                                // table build scratch
        cudaEvent_t ev[2] = {nullptr, nullptr};        // around each build, for its device time
    } builders[2];
    uint64_t lru_clock = 0, resident = 0, batch_seq = 0;
    void *arena = nullptr;                             // table memory when there is a budget
    size_t arena_bytes = 0;
    std::map<size_t, size_t> free_by_off;              // the arena's holes: offset -> size
    std::multimap<size_t, size_t> free_by_size;        // size -> offset
    scr_server_stats stats = {};
    // screener buffers of the plain path
    DevBuf mask_dev, list_dev, small_dev;
    DevBuf keys_host, small_host;                      // pinned
    uint64_t list_dev_cap = 0;
    // batched path: small screens go on a higher-priority stream so they do not
    // queue behind large ones; mapped pinned staging buffers (count | keys) and
    // events are pooled and reused
    cudaStream_t st_small = nullptr;
    std::vector<cudaEvent_t> free_events;
    std::multimap<size_t, void *> free_stage;          // bytes -> mapped pinned buffer
    std::vector<std::pair<void *, size_t>> all_stage;  // every staging buffer, freed at destroy
};

namespace {

int grow_dev(scr_server *s, DevBuf &b, size_t bytes, cudaStream_t st) {
    if (b.bytes >= bytes)
        return SCR_OK;
    if (b.p) {
        cudaStreamSynchronize(st);
        dev_free(s->ctx, b.p, b.bytes, st);
        b.p = nullptr;
        b.bytes = 0;
    }
    bytes = std::max<size_t>(bytes, 4096);
    int rc = dev_alloc(s->ctx, bytes, st, &b.p);
    if (rc)
        return rc;
    b.bytes = bytes;
    return SCR_OK;
}

int grow_host(DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes)
        return SCR_OK;
    if (b.p)
        cudaFreeHost(b.p);
    b.p = nullptr;
    b.bytes = 0;
    bytes = std::max<size_t>(bytes, 4096);
    if (cudaMallocHost(&b.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(SCR_ENOMEM, "pinned host allocation of %zu bytes failed", bytes);
    }
    b.bytes = bytes;
    return SCR_OK;
}

template <class T>
T *device_view(void *host) {   // device address of mapped pinned host memory
    void *d = nullptr;
    if (cudaHostGetDevicePointer(&d, host, 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (T *)d;
}

// Finish a request (server lock held): stamp, release the image, wake waiters.
void complete(scr_server *s, SrvRequest *r, int status) {
    r->res.status = status;
    r->res.done_ns = now_ns();
    r->done = true;
    s->done_q.push_back(r->id);
    SrvImage *im = r->img;
    if (--im->refs == 0 && im->forgotten && !im->building) {
        s->dropped.push_back(im);
        s->cv_build.notify_one();
    }
    s->cv_done.notify_all();
}

// ---------------------------------------------------------------------------
// builder
//
// With a table budget, table memory comes from one device arena reserved when
// the server starts (the budget plus 1/16 for fragmentation) and is handed out
// best-fit by host bookkeeping, so building and evicting tables make no device
// allocation.  Without a budget every table is its own allocation.
// ---------------------------------------------------------------------------

constexpr size_t kArenaAlign = 256;

bool arena_alloc(scr_server *s, size_t need, void **block) {   // lock held
    auto it = s->free_by_size.lower_bound(need);
    if (it == s->free_by_size.end())
        return false;
    const size_t size = it->first, off = it->second;
    s->free_by_size.erase(it);
    s->free_by_off.erase(off);
    if (size > need) {
        s->free_by_off[off + need] = size - need;
        s->free_by_size.emplace(size - need, off + need);
    }
    *block = (char *)s->arena + off;
    return true;
}

void arena_release(scr_server *s, void *block, size_t size) {   // lock held; coalesces neighbours
    size_t off = (size_t)((char *)block - (char *)s->arena);
    auto erase_size = [&](size_t o, size_t sz) {
        auto r = s->free_by_size.equal_range(sz);
        for (auto i = r.first; i != r.second; ++i)
            if (i->second == o) {
                s->free_by_size.erase(i);
                return;
            }
    };
    auto next = s->free_by_off.lower_bound(off);
    if (next != s->free_by_off.end() && next->first == off + size) {
        size += next->second;
        erase_size(next->first, next->second);
        next = s->free_by_off.erase(next);
    }
    if (next != s->free_by_off.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            off = prev->first;
            size += prev->second;
            erase_size(prev->first, prev->second);
            s->free_by_off.erase(prev);
        }
    }
    s->free_by_off[off] = size;
    s->free_by_size.emplace(size, off);
}

// Take the tables off an image (lock held); without an arena their block is
// returned in to_free, to be freed without the lock.
void retire_tables(scr_server *s, SrvImage *im, std::vector<std::pair<size_t, void *>> *to_free) {
    scr_tables *t = im->t;
    im->t = nullptr;
    s->resident -= t->bytes;
    if (s->arena)
        arena_release(s, t->base, t->bytes);
    else if (to_free)
        to_free->push_back({t->bytes, t->base});
    delete t;
}

// Admission by the table budget (server lock held): room for `need` bytes,
// made by evicting the least recently used unpinned tables (also when the
// budget allows but the arena has no hole that large).  Waits for running
// screens to release their pins when only pinned tables stand in the way.  On
// success `need` is charged to resident and *block is the arena block (null
// without an arena: the caller allocates).
int admit(scr_server *s, std::unique_lock<std::mutex> &lk, SrvImage *im, uint64_t need,
          std::vector<std::pair<size_t, void *>> &to_free, void **block) {
    const uint64_t budget = s->cfg.table_budget_bytes;
    *block = nullptr;
    if (budget && need > budget)
        return fail(SCR_EBUDGET, "image %lld: its tables (%llu bytes) exceed the table budget (%llu)",
                    (long long)im->id, (unsigned long long)need, (unsigned long long)budget);
    for (;;) {
        if (!budget || s->resident + need <= budget) {
            if (!s->arena || arena_alloc(s, need, block)) {
                s->resident += need;
                return SCR_OK;
            }
        }
        std::vector<SrvImage *> cand;
        std::vector<uint64_t> bytes, last;
        std::vector<int32_t> pin;
        for (auto &kv : s->images)
            if (kv.second->t) {
                cand.push_back(kv.second);
                bytes.push_back(kv.second->t->bytes);
                last.push_back(kv.second->last_use);
                pin.push_back(kv.second->pins > 0);
            }
        std::vector<int32_t> v(cand.size() + 1);
        int32_t nv = 0;
        const bool fits = s->resident + need <= budget;   // then only the arena is fragmented
        if (server_lru_victims(bytes.data(), last.data(), pin.data(), (int32_t)cand.size(),
                               fits ? budget : s->resident, budget, fits ? 1 : need, v.data(), &nv) == SCR_OK &&
            nv > 0) {
            for (int k = 0; k < nv; ++k) {
                retire_tables(s, cand[v[k]], &to_free);
                s->stats.evictions++;
            }
            continue;
        }
        // only pinned tables are left to evict: wait for the screener to release some
        s->cv_unpin.wait_for(lk, std::chrono::milliseconds(100));
    }
}

void free_blocks(scr_server *s, const std::vector<std::pair<size_t, void *>> &blocks, cudaStream_t st) {
    for (auto &b : blocks)
        dev_free(s->ctx, b.second, b.first, st);
}

void run_job(scr_server *s, scr_server::Builder &bd, BuildJob j) {
    const int64_t t0 = now_ns();
    SrvImage *im = j.img;
    std::unique_lock<std::mutex> lk(s->mu);
    if (j.req)
        j.req->res.start_ns = t0;
    if (j.req && j.req->kind == kEvict) {
        s->cv_unpin.wait(lk, [&] { return im->pins == 0 || im->forgotten; });
        std::vector<std::pair<size_t, void *>> blocks;
        if (!im->forgotten && im->t) {
            retire_tables(s, im, &blocks);
            s->stats.evictions++;
        }
        s->jobs_in_flight--;
        complete(s, j.req, im->forgotten ? SCR_EEVICTED : SCR_OK);
        s->stats.build_ns += now_ns() - t0;
        s->cv_screen.notify_one();
        lk.unlock();
        free_blocks(s, blocks, bd.st);
        return;
    }
    int rc = SCR_OK;
    std::vector<std::pair<size_t, void *>> to_free;
    uint64_t need = 0;
    void *block = nullptr;
    if (im->forgotten)
        rc = SCR_EEVICTED;
    else if (!im->t) {
        need = (tables_bytes(im->H, im->W, s->cfg.sum_bits, s->cfg.sq_bits) + kArenaAlign - 1) & ~(kArenaAlign - 1);
        rc = admit(s, lk, im, need, to_free, &block);
        if (rc == SCR_OK)
            s->stats.peak_resident_bytes = std::max<uint64_t>(s->stats.peak_resident_bytes, s->resident);
    }
    const bool build = rc == SCR_OK && !im->t;
    std::string err = rc ? last_error() : std::string();
    lk.unlock();
    free_blocks(s, to_free, bd.st);
    int64_t t_copy = 0, t_alloc = 0, t_run = 0, t_gpu = 0;
    scr_tables *t = nullptr;
    if (build) {
        int64_t ta = now_ns();
        if ((rc = grow_dev(s, bd.img, (size_t)im->H * im->W, bd.st)) == SCR_OK) {
            cudaError_t e = im->pitch == im->W   // contiguous rows: one plain copy
                                ? cudaMemcpyAsync(bd.img.p, im->host, (size_t)im->H * im->W, cudaMemcpyHostToDevice,
                                                  bd.st)
                                : cudaMemcpy2DAsync(bd.img.p, im->W, im->host, im->pitch, im->W, im->H,
                                                    cudaMemcpyHostToDevice, bd.st);
            if (e != cudaSuccess)
                rc = fail(SCR_ECUDA, "image copy: %s", cudaGetErrorString(e));
        }
        const int64_t tb = now_ns();
        t_copy = tb - ta;
        if (rc == SCR_OK && !block)
            rc = dev_alloc(s->ctx, need, bd.st, &block);
        if (rc == SCR_OK)
            rc = grow_dev(s, bd.scratch, TableScratch::bytes(im->H, im->W, s->cfg.sum_bits, s->cfg.sq_bits), bd.st);
        const int64_t tc = now_ns();
        t_alloc = tc - tb;
        if (rc == SCR_OK) {
            t = new (std::nothrow) scr_tables();
            if (!t)
                rc = fail(SCR_ENOMEM, "host allocation failed");
        }
        if (rc == SCR_OK) {
            layout_tables(t, block, need, im->H, im->W, s->cfg.sum_bits, s->cfg.sq_bits, bd.st);
            const uint64_t before = s->ctx->launches.load();
            cudaEventRecord(bd.ev[0], bd.st);
            rc = run_build_in(s->ctx, (const uint8_t *)bd.img.p, im->H, im->W, im->W, t, bd.scratch.p, bd.st);
            cudaEventRecord(bd.ev[1], bd.st);
            if (rc == SCR_OK && cudaStreamSynchronize(bd.st) != cudaSuccess)
                rc = fail(SCR_ECUDA, "table build failed");
            float ms = 0;
            if (rc == SCR_OK && cudaEventElapsedTime(&ms, bd.ev[0], bd.ev[1]) == cudaSuccess)
                t_gpu = (int64_t)(ms * 1e6f);
            s->stats.launches += s->ctx->launches.load() - before;
        }
        t_run = now_ns() - tc;
        if (rc)
            err = last_error();
    }
    lk.lock();
    if (build) {
        if (rc == SCR_OK && !im->forgotten) {
            im->t = t;
            if (im->builds++)
                s->stats.rebuilds++;
            s->stats.builds++;
        } else {   // failed, or dropped while building: give the block back
            if (rc == SCR_OK)
                rc = SCR_EEVICTED;
            delete t;
            s->resident -= need;
            if (block && s->arena)
                arena_release(s, block, need);
            else if (block)
                to_free.push_back({need, block});
        }
    }
    if (rc == SCR_OK)
        im->last_use = ++s->lru_clock;
    im->building = false;
    s->jobs_in_flight--;
    for (SrvRequest *w : im->waiting) {
        if (rc == SCR_OK) {
            w->res.built = build;
            im->pins++;
            s->ready.push_back(w);
        } else {
            complete(s, w, rc);
        }
    }
    im->waiting.clear();
    if (j.req) {
        j.req->res.built = build && rc == SCR_OK;
        complete(s, j.req, rc);
    }
    s->stats.build_ns += now_ns() - t0;
    s->stats.build_copy_ns += t_copy;
    s->stats.build_alloc_ns += t_alloc;
    s->stats.build_run_ns += t_run;
    s->stats.build_gpu_ns += t_gpu;
    if (rc && !err.empty())
        fail(rc, "%s", err.c_str());
    s->cv_screen.notify_one();
    std::vector<std::pair<size_t, void *>> late;
    late.swap(to_free);
    lk.unlock();
    free_blocks(s, late, bd.st);
}

void builder_main(scr_server *s, scr_server::Builder *bd) {
    cudaSetDevice(s->ctx->device);
    for (;;) {
        BuildJob j = {nullptr, nullptr};
        std::vector<SrvImage *> dropped;
        std::vector<std::pair<size_t, void *>> blocks;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_build.wait(lk, [&] { return s->stop_builder || !s->jobs.empty() || !s->dropped.empty(); });
            dropped.swap(s->dropped);
            for (SrvImage *im : dropped)
                if (im->t)
                    retire_tables(s, im, &blocks);
            if (!s->jobs.empty()) {
                j = s->jobs.front();
                s->jobs.pop_front();
            }
        }
        for (SrvImage *im : dropped)
            delete im;
        free_blocks(s, blocks, bd->st);
        if (j.img)
            run_job(s, *bd, j);
        else if (dropped.empty()) {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->stop_builder && s->jobs.empty())
                break;
        }
    }
}

// ---------------------------------------------------------------------------
// screener
// ---------------------------------------------------------------------------

void deliver(SrvRequest *r, const uint64_t *keys, uint64_t count) {
    r->res.count = count;
    const uint64_t k = std::min(count, r->list_cap);
    if (k && r->list_host)
        memcpy(r->list_host, keys, k * 8);
    r->res.status = count > r->list_cap ? SCR_EOVERFLOW : SCR_OK;
}

// Keys a request's list gets through the staging area; longer lists get the
// rest from the device after the run.
constexpr uint64_t kStageKeys = 1ull << 22;

uint64_t mask_words_of(const SrvRequest *r) {
    return (uint64_t)r->p.n_scales * r->img->H * ((r->img->W + 31) / 32);
}

// Work of one screen, in candidate slots (scales x pixels): orders a batch
// shortest first and picks the stream lane.
uint64_t cost_of(const SrvRequest *r) { return (uint64_t)r->p.n_scales * r->img->H * r->img->W; }

// A screen of at most 2^small_log2 candidate slots (default 2^24) takes the
// priority lane; at most max_inflight screens (default 64) and 4 GiB of their
// masks are enqueued and not yet retired (one screen larger than that runs alone).
uint64_t small_cost(const scr_server *s) { return 1ull << (s->cfg.small_log2 ? s->cfg.small_log2 : 24); }
size_t max_inflight(const scr_server *s) { return s->cfg.max_inflight ? (size_t)s->cfg.max_inflight : 64; }
constexpr uint64_t kInflightMaskBytes = 4ull << 30;

// One screen of the batched path from enqueue to retirement.
struct Inflight {
    SrvRequest *r = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    void *mask = nullptr;
    size_t mask_bytes = 0;
    void *stage = nullptr;        // mapped pinned: count | staged keys
    size_t stage_bytes = 0;
    uint64_t staged_cap = 0;
};

int stage_get(scr_server *s, size_t bytes, void **p, size_t *got) {
    auto it = s->free_stage.lower_bound(bytes);
    if (it != s->free_stage.end()) {
        *p = it->second;
        *got = it->first;
        s->free_stage.erase(it);
        return SCR_OK;
    }
    size_t sz = 64 << 10;
    while (sz < bytes)
        sz <<= 1;
    if (cudaHostAlloc(p, sz, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(SCR_ENOMEM, "mapped host allocation of %zu bytes failed", sz);
    }
    s->all_stage.emplace_back(*p, sz);
    *got = sz;
    return SCR_OK;
}

void release_inflight(scr_server *s, Inflight &f) {
    if (f.mask)
        dev_free(s->ctx, f.mask, f.mask_bytes, f.st);   // stream-ordered: after the screen's kernels
    if (f.stage)
        s->free_stage.emplace(f.stage_bytes, f.stage);
    if (f.ev)
        s->free_events.push_back(f.ev);
    f.mask = f.stage = nullptr;
    f.ev = nullptr;
}

// Enqueue one screen: the single-image screening kernel writes its mask (a
// stream-ordered allocation from the context's pool), the compaction writes its
// count and first keys into mapped host memory, then the screen's event.
// Nothing waits for the device.
int enqueue_screen(scr_server *s, Inflight &f) {
    SrvRequest *r = f.r;
    const uint64_t words = mask_words_of(r);
    f.st = cost_of(r) <= small_cost(s) ? s->st_small : s->st;
    f.staged_cap = std::min(r->list_cap, kStageKeys);
    int rc;
    if (s->free_events.empty()) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return fail(SCR_ECUDA, "event creation failed");
        }
        s->free_events.push_back(ev);
    }
    f.ev = s->free_events.back();
    s->free_events.pop_back();
    if ((rc = stage_get(s, 8 + f.staged_cap * 8, &f.stage, &f.stage_bytes)))
        return rc;
    f.mask_bytes = (size_t)std::max<uint64_t>(words, 1) * 4;
    if ((rc = dev_alloc(s->ctx, f.mask_bytes, f.st, &f.mask))) {
        f.mask = nullptr;
        return rc;
    }
    uint64_t *dst = device_view<uint64_t>(f.stage);
    if (!dst)
        return fail(SCR_ECUDA, "no device address for the mapped staging area");
    const uint64_t before = s->ctx->launches.load();
    if ((rc = screen_features(s->ctx, r->img->t, r->tm, &r->p, (uint32_t *)f.mask, words, (scr_stream)f.st)) ||
        (rc = compact_mask(s->ctx, (const uint32_t *)f.mask, r->p.n_scales, r->img->H, r->img->W,
                           f.staged_cap ? dst + 1 : nullptr, f.staged_cap, dst, (scr_stream)f.st)))
        return rc;
    s->stats.launches += s->ctx->launches.load() - before;
    CUDA_TRY(cudaEventRecord(f.ev, f.st));
    return SCR_OK;
}

// The screen's event has completed: hand the caller its list (a list longer
// than the staging area is compacted again in full from the mask).
int finish_screen(scr_server *s, Inflight &f) {
    SrvRequest *r = f.r;
    const uint64_t *stage = (const uint64_t *)f.stage;
    const uint64_t count = stage[0], m = std::min(count, r->list_cap);
    const uint64_t staged = std::min(m, f.staged_cap);
    if (staged && r->list_host)
        memcpy(r->list_host, stage + 1, staged * 8);
    if (m > staged) {
        int rc;
        if ((rc = grow_dev(s, s->list_dev, (size_t)m * 8, f.st)) || (rc = grow_dev(s, s->small_dev, 64, f.st)))
            return rc;
        if ((rc = compact_mask(s->ctx, (const uint32_t *)f.mask, r->p.n_scales, r->img->H, r->img->W,
                               (uint64_t *)s->list_dev.p, m, (uint64_t *)s->small_dev.p, (scr_stream)f.st)))
            return rc;
        CUDA_TRY(cudaMemcpyAsync(r->list_host, s->list_dev.p, m * 8, cudaMemcpyDeviceToHost, f.st));
        CUDA_TRY(cudaStreamSynchronize(f.st));
        s->list_dev_cap = s->list_dev.bytes / 8;
    }
    r->res.count = count;
    r->res.status = count > r->list_cap ? SCR_EOVERFLOW : SCR_OK;
    return SCR_OK;
}

// One screen with the plain single-image launches.
int run_plain(scr_server *s, SrvRequest *r) {
    const SrvImage *im = r->img;
    const int S = r->p.n_scales;
    const uint64_t words = (uint64_t)S * im->H * ((im->W + 31) / 32);
    int rc;
    if ((rc = grow_dev(s, s->mask_dev, words * 4, s->st)) || (rc = grow_dev(s, s->small_dev, 64, s->st)) ||
        (rc = grow_host(s->small_host, 64)))
        return rc;
    s->stats.mask_bytes = s->mask_dev.bytes;
    if (!s->list_dev_cap) {
        if ((rc = grow_dev(s, s->list_dev, (size_t)8 << 20, s->st)))
            return rc;
        s->list_dev_cap = s->list_dev.bytes / 8;
    }
    uint64_t *cnt_dev = (uint64_t *)s->small_dev.p, *cnt_host = (uint64_t *)s->small_host.p;
    const uint64_t before = s->ctx->launches.load();
    if ((rc = screen_features(s->ctx, im->t, r->tm, &r->p, (uint32_t *)s->mask_dev.p, words, (scr_stream)s->st)))
        return rc;
    for (int pass = 0;; ++pass) {
        if ((rc = compact_mask(s->ctx, (const uint32_t *)s->mask_dev.p, S, im->H, im->W, (uint64_t *)s->list_dev.p,
                               s->list_dev_cap, cnt_dev, (scr_stream)s->st)))
            return rc;
        CUDA_TRY(cudaMemcpyAsync(cnt_host, cnt_dev, 8, cudaMemcpyDeviceToHost, s->st));
        CUDA_TRY(cudaStreamSynchronize(s->st));
        const uint64_t want = std::min(cnt_host[0], r->list_cap);
        if (want <= s->list_dev_cap || pass)
            break;
        if ((rc = grow_dev(s, s->list_dev, (size_t)(((want >> 20) + 1) << 20) * 8, s->st)))
            return rc;
        s->list_dev_cap = s->list_dev.bytes / 8;
    }
    s->stats.launches += s->ctx->launches.load() - before;
    const uint64_t count = cnt_host[0];
    const uint64_t k = std::min(count, r->list_cap);
    if ((rc = grow_host(s->keys_host, (size_t)std::max<uint64_t>(k, 1) * 8)))
        return rc;
    if (k) {
        CUDA_TRY(cudaMemcpyAsync(s->keys_host.p, s->list_dev.p, k * 8, cudaMemcpyDeviceToHost, s->st));
        CUDA_TRY(cudaStreamSynchronize(s->st));
    }
    deliver(r, (const uint64_t *)s->keys_host.p, count);
    return SCR_OK;
}

// Sort newly submitted screens (server lock held): to the ready list, pinning
// their tables, or to their image's waiting list, asking for a rebuild when
// none is under way.
void sort_pending(scr_server *s) {
    while (!s->pending.empty()) {
        SrvRequest *r = s->pending.front();
        s->pending.pop_front();
        SrvImage *im = r->img;
        if (im->forgotten) {
            complete(s, r, SCR_EEVICTED);
            continue;
        }
        if (im->t && !im->building) {
            im->pins++;
            s->ready.push_back(r);
        } else {
            im->waiting.push_back(r);
            if (!im->building) {
                im->building = true;
                s->jobs.push_back({im, nullptr});
                s->jobs_in_flight++;
                s->cv_build.notify_one();
            }
        }
    }
}

bool drained(const scr_server *s) {
    return s->pending.empty() && s->ready.empty() && s->jobs.empty() && s->jobs_in_flight == 0;
}

// Release a finished batch's requests (takes the server lock).
void retire(scr_server *s, const std::vector<SrvRequest *> &batch, int64_t t0) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.batches++;
    s->stats.screen_ns += now_ns() - t0;
    for (SrvRequest *r : batch) {
        r->img->pins--;
        r->img->last_use = ++s->lru_clock;
        complete(s, r, r->res.status);
    }
    s->cv_unpin.notify_all();
}

// Release one screen of the batched path (server lock held).
void retire_one(scr_server *s, SrvRequest *r) {
    r->img->pins--;
    r->img->last_use = ++s->lru_clock;
    complete(s, r, r->res.status);
}

// Plain mode: serve each screen with its own launches and wait for it.
void plain_loop(scr_server *s) {
    for (;;) {
        std::vector<SrvRequest *> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_screen.wait(lk, [&] {
                return (!s->hold && (!s->pending.empty() || !s->ready.empty())) || (s->stop && drained(s));
            });
            if (s->stop && drained(s))
                return;
            sort_pending(s);
            const size_t lim = s->cfg.max_batch > 0 ? (size_t)s->cfg.max_batch : s->ready.size();
            const size_t take = std::min(lim, s->ready.size());
            batch.assign(s->ready.begin(), s->ready.begin() + take);
            s->ready.erase(s->ready.begin(), s->ready.begin() + take);
        }
        if (batch.empty())
            continue;
        const int64_t t0 = now_ns();
        const uint64_t seq = ++s->batch_seq;
        for (SrvRequest *r : batch) {
            r->res.start_ns = t0;
            r->res.batch = seq;
            r->res.batch_size = (int32_t)batch.size();
        }
        for (SrvRequest *r : batch) {
            const int rc = run_plain(s, r);
            if (rc)
                r->res.status = rc;
        }
        retire(s, batch, t0);
    }
}

// Batched mode (continuous batching): whenever screens are ready and there is
// room in flight, take them all (at most max_batch) as one batch, order it
// shortest first and enqueue every screen without waiting (small ones on the
// priority stream, so they overtake large ones already on the device); retire
// each screen as soon as its own event completes, while later batches are
// being admitted.  Room in flight: max_inflight screens and kInflightMaskBytes
// of masks (one screen larger than that runs alone).
void batched_loop(scr_server *s) {
    std::vector<Inflight> flying;
    uint64_t flying_mask = 0;
    for (;;) {
        std::vector<SrvRequest *> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto room = [&] { return flying.size() < max_inflight(s) && flying_mask < kInflightMaskBytes; };
            auto can_take = [&] { return !s->hold && room() && (!s->pending.empty() || !s->ready.empty()); };
            if (flying.empty()) {
                s->cv_screen.wait(lk, [&] { return can_take() || (s->stop && drained(s)); });
                if (s->stop && drained(s))
                    return;
            } else if (!can_take()) {   // poll the screens in flight while waiting for arrivals
                const int64_t w0 = now_ns();
                s->cv_screen.wait_for(lk, std::chrono::microseconds(10), can_take);
                s->stats.wait_ns += now_ns() - w0;
                s->stats.screen_ns += now_ns() - w0;
            }
            if (can_take()) {
                sort_pending(s);
                const size_t lim = s->cfg.max_batch > 0 ? (size_t)s->cfg.max_batch : s->ready.size();
                uint64_t m = flying_mask;
                size_t take = 0;
                while (take < std::min(lim, s->ready.size()) && flying.size() + take < max_inflight(s)) {
                    const uint64_t b = mask_words_of(s->ready[take]) * 4;
                    if ((take || !flying.empty()) && m + b > kInflightMaskBytes)
                        break;
                    m += b;
                    ++take;
                }
                batch.assign(s->ready.begin(), s->ready.begin() + take);
                s->ready.erase(s->ready.begin(), s->ready.begin() + take);
            }
        }
        if (!batch.empty()) {
            const int64_t t0 = now_ns();
            const uint64_t seq = ++s->batch_seq;
            std::stable_sort(batch.begin(), batch.end(),
                             [](const SrvRequest *a, const SrvRequest *b) { return cost_of(a) < cost_of(b); });
            std::vector<SrvRequest *> failed;
            for (SrvRequest *r : batch) {
                r->res.start_ns = t0;
                r->res.batch = seq;
                r->res.batch_size = (int32_t)batch.size();
                Inflight f;
                f.r = r;
                const int rc = enqueue_screen(s, f);
                if (rc) {
                    // nothing of this screen is left on the device past this point
                    if (f.st)
                        cudaStreamSynchronize(f.st);
                    release_inflight(s, f);
                    r->res.status = rc;
                    failed.push_back(r);
                    continue;
                }
                flying_mask += f.mask_bytes;
                flying.push_back(f);
            }
            s->stats.batches++;
            s->stats.plan_ns += now_ns() - t0;
            s->stats.screen_ns += now_ns() - t0;
            if (!failed.empty()) {
                std::lock_guard<std::mutex> lk(s->mu);
                for (SrvRequest *r : failed)
                    retire_one(s, r);
                s->cv_unpin.notify_all();
            }
        }
        // retire every screen whose event has completed (out of order across the lanes)
        std::vector<SrvRequest *> done;
        const int64_t c0 = now_ns();
        for (size_t k = 0; k < flying.size();) {
            Inflight &f = flying[k];
            const cudaError_t q = cudaEventQuery(f.ev);
            if (q == cudaErrorNotReady) {
                cudaGetLastError();
                ++k;
                continue;
            }
            int rc = q == cudaSuccess ? finish_screen(s, f) : fail(SCR_ECUDA, "screen: %s", cudaGetErrorString(q));
            if (rc)
                f.r->res.status = rc;
            cudaGetLastError();
            flying_mask -= f.mask_bytes;
            release_inflight(s, f);
            done.push_back(f.r);
            flying[k] = flying.back();
            flying.pop_back();
        }
        if (!done.empty()) {
            s->stats.copy_ns += now_ns() - c0;
            s->stats.screen_ns += now_ns() - c0;
            std::lock_guard<std::mutex> lk(s->mu);
            for (SrvRequest *r : done)
                retire_one(s, r);
            s->cv_unpin.notify_all();
        }
    }
}

void screener_main(scr_server *s) {
    cudaSetDevice(s->ctx->device);
    if (s->cfg.mode == SCR_SERVE_BATCHED)
        batched_loop(s);
    else
        plain_loop(s);
}

int submit(scr_server *s, SrvRequest *r, uint64_t *request_id) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        delete r;
        return fail(SCR_EINVAL, "server is shutting down");
    }
    r->id = s->next_req++;
    r->img->refs++;
    s->reqs[r->id] = r;
    s->stats.requests++;
    if (request_id)
        *request_id = r->id;
    if (r->kind == kScreen) {
        s->pending.push_back(r);
        s->cv_screen.notify_one();
    } else {   // uploads and evictions go straight to the builder, held or not
        if (r->kind == kUpload)
            r->img->building = true;
        s->jobs.push_back({r->img, r});
        s->jobs_in_flight++;
        s->cv_build.notify_one();
    }
    return SCR_OK;
}

SrvImage *find_image(scr_server *s, int64_t id) {   // server lock held
    auto it = s->images.find(id);
    return it == s->images.end() ? nullptr : it->second;
}

}  // namespace

namespace scr_rt {
// a context's servers are destroyed by screen_shutdown
void destroy_servers(scr_ctx *c) {
    std::vector<scr_server *> v;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        v.assign(c->servers.begin(), c->servers.end());
    }
    for (scr_server *s : v)
        server_destroy(s);
}
}  // namespace scr_rt

extern "C" {

int64_t server_clock_ns(void) { return now_ns(); }

int server_lru_victims(const uint64_t *bytes, const uint64_t *last_use, const int32_t *pinned, int32_t n,
                       uint64_t resident, uint64_t budget, uint64_t need, int32_t *victims, int32_t *n_victims) {
    if (!n_victims || n < 0 || (n > 0 && (!bytes || !last_use || !pinned || !victims)))
        return fail(SCR_EINVAL, "null argument");
    *n_victims = 0;
    if (resident + need <= budget)
        return SCR_OK;
    std::vector<int32_t> order;
    for (int32_t i = 0; i < n; ++i)
        if (!pinned[i])
            order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return last_use[a] < last_use[b]; });
    uint64_t cur = resident;
    int32_t k = 0;
    for (int32_t i : order) {
        if (cur + need <= budget)
            break;
        cur -= std::min(cur, bytes[i]);
        victims[k++] = i;
    }
    if (cur + need > budget)
        return fail(SCR_EBUDGET, "evicting every unpinned table leaves %llu + %llu bytes above the budget %llu",
                    (unsigned long long)cur, (unsigned long long)need, (unsigned long long)budget);
    *n_victims = k;
    return SCR_OK;
}

int server_create(scr_ctx *c, const scr_server_config *cfg, scr_server **out) {
    int rc;
    if ((rc = check_ctx(c)))
        return rc;
    if (!cfg || !out)
        return fail(SCR_EINVAL, "null config or out-pointer");
    if ((cfg->sum_bits != 32 && cfg->sum_bits != 64) || (cfg->sq_bits != 32 && cfg->sq_bits != 64))
        return fail(SCR_EINVAL, "table widths must be 32 or 64 bits");
    if (cfg->mode != SCR_SERVE_BATCHED && cfg->mode != SCR_SERVE_PLAIN)
        return fail(SCR_EINVAL, "unknown serving mode %d", cfg->mode);
    if (cfg->small_log2 < 0 || cfg->small_log2 > 40 || cfg->max_inflight < 0 || cfg->max_inflight > 4096 ||
        cfg->max_batch < 0)
        return fail(SCR_EINVAL, "small_log2 must be in [0, 40], max_inflight in [0, 4096], max_batch >= 0");
    *out = nullptr;
    DeviceGuard dg(c->device);
    auto *s = new (std::nothrow) scr_server();
    if (!s)
        return fail(SCR_ENOMEM, "host allocation failed");
    s->ctx = c;
    s->cfg = *cfg;
    s->hold = cfg->start_held != 0;
    // table builds go first when they and screening kernels wait for the same
    // SMs; small screens come next, large screens last
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    const int prio_small = prio_hi < prio_lo ? prio_hi + 1 : prio_hi;
    cudaError_t e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithPriority(&s->st_small, cudaStreamNonBlocking, prio_small);
    for (auto &bd : s->builders)
        if (e == cudaSuccess)
            e = cudaStreamCreateWithPriority(&bd.st, cudaStreamNonBlocking, prio_hi);
    auto drop_streams = [&] {
        for (cudaStream_t q : {s->st, s->st_small})
            if (q)
                cudaStreamDestroy(q);
        for (auto &bd : s->builders)
            if (bd.st)
                cudaStreamDestroy(bd.st);
    };
    if (e != cudaSuccess) {
        drop_streams();
        delete s;
        return fail(SCR_ECUDA, "stream creation: %s", cudaGetErrorString(e));
    }
    if (cfg->table_budget_bytes) {
        const size_t want = (size_t)cfg->table_budget_bytes + (size_t)(cfg->table_budget_bytes >> 4);
        if ((rc = dev_alloc(c, (want + kArenaAlign - 1) & ~(kArenaAlign - 1), s->st, &s->arena))) {
            drop_streams();
            delete s;
            return rc;
        }
        s->arena_bytes = (want + kArenaAlign - 1) & ~(kArenaAlign - 1);
        s->free_by_off[0] = s->arena_bytes;
        s->free_by_size.emplace(s->arena_bytes, 0);
        cudaStreamSynchronize(s->st);
    }
    for (auto &bd : s->builders) {
        cudaEventCreate(&bd.ev[0]);
        cudaEventCreate(&bd.ev[1]);
        bd.th = std::thread(builder_main, s, &bd);
    }
    s->screener = std::thread(screener_main, s);
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->servers.insert(s);
    }
    *out = s;
    return SCR_OK;
}

int server_upload(scr_server *s, const uint8_t *img_host, int32_t H, int32_t W, int64_t pitch, int32_t borrow,
                  int64_t arrival_ns, int64_t *image_id, uint64_t *request_id) {
    if (!s || !img_host || !image_id)
        return fail(SCR_EINVAL, "null server, image or id out-pointer");
    if (H < 1 || W < 1 || H > 65535 || W > 65535 || pitch < W)
        return fail(SCR_EINVAL, "image %d x %d (pitch %lld) outside 1..65535", H, W, (long long)pitch);
    auto *im = new (std::nothrow) SrvImage();
    auto *r = new (std::nothrow) SrvRequest();
    if (!im || !r) {
        delete im;
        delete r;
        return fail(SCR_ENOMEM, "host allocation failed");
    }
    im->H = H;
    im->W = W;
    if (borrow) {
        im->host = img_host;
        im->pitch = pitch;
    } else {
        try {
            im->own.resize((size_t)H * W);
        } catch (...) {
            delete im;
            delete r;
            return fail(SCR_ENOMEM, "host copy of %d x %d failed", H, W);
        }
        for (int y = 0; y < H; ++y)
            memcpy(im->own.data() + (size_t)y * W, img_host + (size_t)y * pitch, W);
        im->host = im->own.data();
        im->pitch = W;
    }
    r->kind = kUpload;
    r->img = im;
    r->res.kind = kUpload;
    r->res.arrival_ns = arrival_ns ? arrival_ns : now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        im->id = s->next_image++;
        s->images[im->id] = im;
        s->stats.uploads++;
    }
    *image_id = im->id;
    return submit(s, r, request_id);
}

int server_screen(scr_server *s, int64_t image_id, const scr_tmpl *tm, const scr_params *p, uint64_t *list_host,
                  uint64_t list_cap, int64_t arrival_ns, uint64_t *request_id) {
    if (!s || !tm || !p)
        return fail(SCR_EINVAL, "null server, template or params");
    if (list_cap && !list_host)
        return fail(SCR_EINVAL, "null list buffer with list_cap %llu", (unsigned long long)list_cap);
    int rc = validate_params(p);
    if (rc)
        return rc;
    if ((p->features & SCR_F_GRAD) && !(tm->features & SCR_F_GRAD))
        return fail(SCR_EINVAL, "template features were computed without SCR_F_GRAD");
    if (p->features & SCR_F_PREWITT)
        return fail(SCR_EUNSUPPORTED, "the serving loop has no Prewitt test");
    auto *r = new (std::nothrow) SrvRequest();
    if (!r)
        return fail(SCR_ENOMEM, "host allocation failed");
    r->kind = kScreen;
    r->tm = tm;
    r->p = *p;
    r->radii.assign(p->radii, p->radii + p->n_scales);
    r->p.radii = r->radii.data();
    r->list_host = list_host;
    r->list_cap = list_cap;
    r->res.kind = kScreen;
    r->res.arrival_ns = arrival_ns ? arrival_ns : now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        SrvImage *im = find_image(s, image_id);
        if (!im) {
            delete r;
            return fail(SCR_EEVICTED, "image %lld is unknown or was forgotten", (long long)image_id);
        }
        r->img = im;
        s->stats.screens++;
    }
    return submit(s, r, request_id);
}

int server_evict(scr_server *s, int64_t image_id, uint64_t *request_id) {
    if (!s)
        return fail(SCR_EINVAL, "null server");
    auto *r = new (std::nothrow) SrvRequest();
    if (!r)
        return fail(SCR_ENOMEM, "host allocation failed");
    r->kind = kEvict;
    r->res.kind = kEvict;
    r->res.arrival_ns = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        SrvImage *im = find_image(s, image_id);
        if (!im) {
            delete r;
            return fail(SCR_EEVICTED, "image %lld is unknown or was forgotten", (long long)image_id);
        }
        r->img = im;
    }
    return submit(s, r, request_id);
}

int server_forget(scr_server *s, int64_t image_id) {
    if (!s)
        return fail(SCR_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    SrvImage *im = find_image(s, image_id);
    if (!im)
        return fail(SCR_EEVICTED, "image %lld is unknown or was forgotten", (long long)image_id);
    s->images.erase(image_id);
    im->forgotten = true;
    if (im->refs == 0 && !im->building) {
        s->dropped.push_back(im);   // the builder frees it
        s->cv_build.notify_one();
    }
    s->cv_unpin.notify_all();
    return SCR_OK;
}

int server_wait(scr_server *s, uint64_t request_id, int64_t timeout_us, scr_request_result *out) {
    if (!s || !out)
        return fail(SCR_EINVAL, "null server or result");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end())
        return fail(SCR_EINVAL, "unknown or collected request %llu", (unsigned long long)request_id);
    SrvRequest *r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_us < 0)
        s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
        return fail(SCR_ETIMEOUT, "request %llu still pending", (unsigned long long)request_id);
    *out = r->res;
    s->reqs.erase(it);
    delete r;
    return SCR_OK;
}

int server_next(scr_server *s, int64_t timeout_us, uint64_t *request_id, scr_request_result *out) {
    if (!s || !out || !request_id)
        return fail(SCR_EINVAL, "null server, id or result");
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {   // drop ids that server_wait collected already
        while (!s->done_q.empty() && !s->reqs.count(s->done_q.front()))
            s->done_q.pop_front();
        return !s->done_q.empty();
    };
    if (timeout_us < 0)
        s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
        return fail(SCR_ETIMEOUT, "no request completed in time");
    const uint64_t id = s->done_q.front();
    s->done_q.pop_front();
    auto it = s->reqs.find(id);
    *request_id = id;
    *out = it->second->res;
    delete it->second;
    s->reqs.erase(it);
    return SCR_OK;
}

int server_hold(scr_server *s, int32_t hold) {
    if (!s)
        return fail(SCR_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    s->hold = hold != 0;
    s->cv_screen.notify_one();
    return SCR_OK;
}

int server_resident(scr_server *s, int64_t image_id, int32_t *resident) {
    if (!s || !resident)
        return fail(SCR_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    SrvImage *im = find_image(s, image_id);
    if (!im)
        return fail(SCR_EEVICTED, "image %lld is unknown or was forgotten", (long long)image_id);
    *resident = im->t != nullptr;
    return SCR_OK;
}

int server_stats(scr_server *s, scr_server_stats *out) {
    if (!s || !out)
        return fail(SCR_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.resident_bytes = s->resident;
    uint64_t ri = 0;
    for (auto &kv : s->images)
        ri += kv.second->t != nullptr;
    s->stats.resident_images = ri;
    *out = s->stats;
    return SCR_OK;
}

void server_destroy(scr_server *s) {
    if (!s)
        return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->hold = false;
        s->cv_screen.notify_all();
    }
    if (s->screener.joinable())
        s->screener.join();   // returns once every request is served
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop_builder = true;
        s->cv_build.notify_all();
    }
    for (auto &bd : s->builders)
        if (bd.th.joinable())
            bd.th.join();
    scr_ctx *c = s->ctx;
    DeviceGuard dg(c->device);
    cudaStreamSynchronize(s->st);
    cudaStreamSynchronize(s->st_small);
    for (auto &bd : s->builders)
        cudaStreamSynchronize(bd.st);
    std::vector<std::pair<size_t, void *>> blocks;
    for (auto &kv : s->images) {
        if (kv.second->t)
            retire_tables(s, kv.second, &blocks);
        delete kv.second;
    }
    for (SrvImage *im : s->dropped) {
        if (im->t)
            retire_tables(s, im, &blocks);
        delete im;
    }
    free_blocks(s, blocks, s->st);
    if (s->arena)
        dev_free(c, s->arena, s->arena_bytes, s->st);
    for (auto &kv : s->reqs)
        delete kv.second;
    for (DevBuf *b : {&s->mask_dev, &s->list_dev, &s->small_dev})
        dev_free(c, b->p, b->bytes, s->st);
    for (auto &bd : s->builders) {
        dev_free(c, bd.img.p, bd.img.bytes, bd.st);
        dev_free(c, bd.scratch.p, bd.scratch.bytes, bd.st);
    }
    cudaStreamSynchronize(s->st);
    for (auto &bd : s->builders)
        cudaStreamSynchronize(bd.st);
    for (DevBuf *b : {&s->keys_host, &s->small_host})
        if (b->p)
            cudaFreeHost(b->p);
    for (auto &kv : s->all_stage)
        cudaFreeHost(kv.first);
    for (cudaEvent_t ev : s->free_events)
        cudaEventDestroy(ev);
    cudaStreamDestroy(s->st);
    cudaStreamDestroy(s->st_small);
    for (auto &bd : s->builders) {
        cudaStreamDestroy(bd.st);
        for (cudaEvent_t e : bd.ev)
            if (e)
                cudaEventDestroy(e);
    }
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->servers.erase(s);
    }
    delete s;
}

}  // extern "C"
