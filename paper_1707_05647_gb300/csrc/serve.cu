// Serving loop of include/screen.h.  Two threads per server:
//  - two builders build the tables of uploaded images and rebuild evicted ones
//    from their host copy (each on its own stream), admitting new tables by the
//    table budget: it evicts least recently used tables that no ready or running
//    screen pins, and waits for pins to be released when that is not enough;
//  - the screener takes every screen whose tables are resident whenever it is
//    free (continuous batching) and runs them as one batched launch or as one
//    plain launch pair each, then hands each request its list in the
//    single-image key format.
// Copies and table builds of the builder overlap with the screener's kernels.
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
    // screener buffers: the plain path's, and one set per batched run in flight
    DevBuf mask_dev, list_dev, small_dev;
    DevBuf keys_host, small_host;                      // pinned
    uint64_t list_dev_cap = 0;
    struct Slot {
        DevBuf mask_dev;       // every request's mask planes, one segment each
        DevBuf segs_dev;       // the segments (MaskSeg)
        DevBuf scratch_dev;    // segmented compaction scratch
        DevBuf desc_host;      // pinned copy of the plan and the segments for the upload
        DevBuf out_host;       // mapped pinned: counts[n] | staged keys
        cudaEvent_t done = nullptr;
        bool busy = false;
    } slots[2];
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

int grow_mapped(DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes)
        return SCR_OK;
    if (b.p)
        cudaFreeHost(b.p);
    b.p = nullptr;
    b.bytes = 0;
    bytes = std::max<size_t>(bytes + (bytes >> 2), 1 << 20);
    if (cudaHostAlloc(&b.p, bytes, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(SCR_ENOMEM, "mapped host allocation of %zu bytes failed", bytes);
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

uint64_t seg_words_of(const SrvRequest *r) {   // rounded up to whole compaction chunks
    return (mask_words_of(r) + kCompactChunk - 1) / kCompactChunk * kCompactChunk;
}

struct StageLayout {
    size_t counts, keys, bytes;          // byte offsets in the mapped area
    std::vector<uint64_t> cap, off;      // per request: staged keys and their offset
};

StageLayout stage_layout(const std::vector<SrvRequest *> &scr) {
    StageLayout L;
    L.counts = 0;
    L.keys = (8 * scr.size() + 255) & ~size_t(255);
    uint64_t pos = 0;
    for (SrvRequest *r : scr) {
        const uint64_t c = std::min(r->list_cap, kStageKeys);
        L.cap.push_back(c);
        L.off.push_back(pos);
        pos += c;
    }
    L.bytes = L.keys + pos * 8 + 8;
    return L;
}

// Enqueue one batched run of `scr` on the screener stream using slot `sl`:
// the screening kernel in mask mode writes each (request, scale) plane of a
// zeroed mask buffer (records grouped per (image, star radius), so positions
// and radii shared by several requests are computed once), then one segmented
// compaction writes each request's first keys, in compact_mask's format and
// order, and its count into mapped host memory; then the slot's event.
// Nothing waits for the device.
int launch_batched(scr_server *s, scr_server::Slot &sl, const std::vector<SrvRequest *> &scr) {
    const int n = (int)scr.size();
    std::vector<const scr_tables *> tabs;
    std::unordered_map<SrvImage *, int> idx;
    std::vector<scr_pair> pairs(n);
    std::vector<const scr_tmpl *> tms(n);
    std::vector<scr_params> ps(n);
    std::vector<MaskSeg> segs(n);
    const StageLayout L = stage_layout(scr);
    uint64_t words = 0;
    for (int k = 0; k < n; ++k) {
        SrvRequest *r = scr[k];
        auto it = idx.find(r->img);
        if (it == idx.end()) {
            it = idx.emplace(r->img, (int)tabs.size()).first;
            tabs.push_back(r->img->t);
        }
        pairs[k].image = it->second;
        pairs[k].tmpl = k;
        tms[k] = r->tm;
        ps[k] = r->p;
        MaskSeg &g = segs[k];
        g.word0 = words;
        g.words = mask_words_of(r);
        g.chunk0 = (uint32_t)(words / kCompactChunk);
        g.nchunks = (uint32_t)(seg_words_of(r) / kCompactChunk);
        g.H = r->img->H;
        g.Wwords = (r->img->W + 31) / 32;
        g.cap = L.cap[k];
        g.out0 = L.off[k];
        words += seg_words_of(r);
    }
    const uint64_t nchunks = words / kCompactChunk;
    int rc;
    if ((rc = grow_dev(s, sl.mask_dev, words * 4, s->st)) ||
        (rc = grow_dev(s, sl.segs_dev, (size_t)n * sizeof(MaskSeg), s->st)) ||
        (rc = grow_dev(s, sl.scratch_dev, compact_segments_scratch_bytes(nchunks), s->st)) ||
        (rc = grow_mapped(sl.out_host, L.bytes)))
        return rc;
    s->stats.mask_bytes = s->slots[0].mask_dev.bytes + s->slots[1].mask_dev.bytes;
    char *dout = device_view<char>(sl.out_host.p);
    if (!dout)
        return fail(SCR_ECUDA, "no device address for the mapped staging area");
    scr_batch *b = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->ctx->mu);
        rc = batch_prepare(s->ctx, tabs.data(), (int)tabs.size(), tms.data(), ps.data(), n, pairs.data(), n,
                           (uint64_t *)sl.segs_dev.p, nullptr, nullptr, nullptr, 0, (uint64_t *)sl.segs_dev.p, s->st,
                           &b);
    }
    if (rc)
        return rc;
    for (BRecord &rc_ : b->records)   // each (request, scale) plane of the mask buffer
        rc_.mask_plane = (int64_t)(segs[rc_.pair].word0 + (uint64_t)rc_.s * segs[rc_.pair].H * segs[rc_.pair].Wwords);
    batch_set_shape(b, s->cfg.words_per_warp ? s->cfg.words_per_warp : 4,
                    s->cfg.blocks_per_sm ? s->cfg.blocks_per_sm : 4);
    // Short-lived blocks: each warp takes at most kUnitsPerWarp units and the
    // grid covers the plan, so blocks keep finishing and the builders'
    // higher-priority table builds get SMs while a batch runs.
    {
        constexpr uint32_t kUnitsPerWarp = 4;
        const uint64_t warps = ((uint64_t)b->n_units + kUnitsPerWarp - 1) / kUnitsPerWarp;
        const uint64_t blocks = (warps + kBatchWarpsPerBlock - 1) / kBatchWarpsPerBlock;
        b->grid = (int)std::max<uint64_t>(std::min<uint64_t>(blocks, 1u << 20), (uint64_t)b->grid);
        b->args.units_per_warp = (uint32_t)std::max<uint64_t>(
            1, ((uint64_t)b->n_units + (uint64_t)b->grid * kBatchWarpsPerBlock - 1) /
                   ((uint64_t)b->grid * kBatchWarpsPerBlock));
    }
    b->args.masks = (uint32_t *)sl.mask_dev.p;
    uint64_t launches = 0;
    const size_t seg_at = (b->desc_bytes + 255) & ~size_t(255);
    if ((rc = grow_host(sl.desc_host, seg_at + (size_t)n * sizeof(MaskSeg))) == SCR_OK) {
        pack_plan(b, sl.desc_host.p);
        memcpy((char *)sl.desc_host.p + seg_at, segs.data(), (size_t)n * sizeof(MaskSeg));
        cudaError_t e = cudaMemcpyAsync(b->desc, sl.desc_host.p, b->desc_bytes, cudaMemcpyHostToDevice, s->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sl.segs_dev.p, (char *)sl.desc_host.p + seg_at, (size_t)n * sizeof(MaskSeg),
                                cudaMemcpyHostToDevice, s->st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(sl.mask_dev.p, 0, words * 4, s->st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(b->n_reserved, 0, 16, s->st);   // the kernel's unit counter
        if (e == cudaSuccess && b->n_units > 0 && !b->groups.empty())
            e = launch_batch(b->args, b->wpw, b->grid, s->st, &launches);
        if (e == cudaSuccess)
            e = launch_compact_segments((const uint32_t *)sl.mask_dev.p, (const MaskSeg *)sl.segs_dev.p, n, nchunks,
                                        (uint64_t *)(dout + L.keys), (uint64_t *)(dout + L.counts), sl.scratch_dev.p,
                                        s->st, &launches);
        if (e == cudaSuccess)
            e = cudaEventRecord(sl.done, s->st);
        if (e != cudaSuccess)
            rc = fail(SCR_ECUDA, "batched run: %s", cudaGetErrorString(e));
    }
    s->stats.launches += launches;
    s->ctx->launches += launches;
    {
        std::lock_guard<std::mutex> lk(s->ctx->mu);
        free_batch_on(s->ctx, b, s->st);   // stream-ordered after the run
    }
    return rc;
}

// Wait for a run launched by launch_batched and deliver every request's list.
int finish_batched(scr_server *s, scr_server::Slot &sl, const std::vector<SrvRequest *> &scr) {
    const int64_t t0 = now_ns();
    CUDA_TRY(cudaEventSynchronize(sl.done));
    const int64_t t1 = now_ns();
    s->stats.wait_ns += t1 - t0;
    const StageLayout L = stage_layout(scr);
    const char *out = (const char *)sl.out_host.p;
    const uint64_t *cnt = (const uint64_t *)(out + L.counts);
    const uint64_t *keys = (const uint64_t *)(out + L.keys);
    uint64_t word0 = 0;
    for (size_t k = 0; k < scr.size(); ++k) {
        SrvRequest *r = scr[k];
        const uint64_t c = cnt[k], m = std::min(c, r->list_cap);
        const uint64_t staged = std::min(m, L.cap[k]);
        if (staged && r->list_host)
            memcpy(r->list_host, keys + L.off[k], staged * 8);
        if (m > staged) {   // a list longer than its staging slot: compact the mask again, in full
            int rc;
            if ((rc = grow_dev(s, s->list_dev, (size_t)m * 8, s->st)) || (rc = grow_dev(s, s->small_dev, 64, s->st)))
                return rc;
            if ((rc = compact_mask(s->ctx, (const uint32_t *)sl.mask_dev.p + word0, r->p.n_scales, r->img->H,
                                   r->img->W, (uint64_t *)s->list_dev.p, m, (uint64_t *)s->small_dev.p,
                                   (scr_stream)s->st)))
                return rc;
            CUDA_TRY(cudaMemcpyAsync(r->list_host, s->list_dev.p, m * 8, cudaMemcpyDeviceToHost, s->st));
            CUDA_TRY(cudaStreamSynchronize(s->st));
            s->list_dev_cap = s->list_dev.bytes / 8;
        }
        r->res.count = c;
        r->res.status = c > r->list_cap ? SCR_EOVERFLOW : SCR_OK;
        word0 += seg_words_of(r);
    }
    s->stats.copy_ns += now_ns() - t1;
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

constexpr uint64_t kBatchMaskWords = 1ull << 31;   // 8 GiB of masks per batched run at most

struct Flight {
    std::vector<SrvRequest *> reqs;
    int slot = 0;
    int rc = SCR_OK;
    int64_t t0 = 0;
};

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

// The screener: batched mode keeps up to two runs in flight, so the next batch
// is planned and enqueued while the device still works on the previous one;
// plain mode serves each screen with its own launches and waits for it.
void screener_main(scr_server *s) {
    cudaSetDevice(s->ctx->device);
    std::deque<Flight> flights;
    const bool batched = s->cfg.mode == SCR_SERVE_BATCHED;
    for (;;) {
        std::vector<SrvRequest *> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto can_take = [&] { return !s->hold && (!s->pending.empty() || !s->ready.empty()); };
            if (flights.empty())
                s->cv_screen.wait(lk, [&] { return can_take() || (s->stop && drained(s)); });
            else if (!can_take())   // poll the oldest run while waiting for arrivals
                s->cv_screen.wait_for(lk, std::chrono::microseconds(20), can_take);
            if (flights.empty() && s->stop && drained(s))
                break;
            if (flights.size() < 2 && can_take()) {
                sort_pending(s);
                const size_t lim = s->cfg.max_batch > 0 ? (size_t)s->cfg.max_batch : s->ready.size();
                size_t take = 0;
                uint64_t words = 0;   // the batched path's mask buffer stays below kBatchMaskWords
                while (take < std::min(lim, s->ready.size())) {
                    words += seg_words_of(s->ready[take]);
                    if (take && batched && words > kBatchMaskWords)
                        break;
                    ++take;
                }
                batch.assign(s->ready.begin(), s->ready.begin() + take);
                s->ready.erase(s->ready.begin(), s->ready.begin() + take);
            }
        }
        if (!batch.empty()) {
            const int64_t t0 = now_ns();
            const uint64_t seq = ++s->batch_seq;
            for (SrvRequest *r : batch) {
                r->res.start_ns = t0;
                r->res.batch = seq;
                r->res.batch_size = (int32_t)batch.size();
            }
            if (batched) {
                Flight f;
                f.reqs = std::move(batch);
                f.t0 = t0;
                f.slot = s->slots[0].busy ? 1 : 0;
                s->slots[f.slot].busy = true;
                f.rc = launch_batched(s, s->slots[f.slot], f.reqs);
                s->stats.plan_ns += now_ns() - t0;
                flights.push_back(std::move(f));
                continue;
            }
            for (SrvRequest *r : batch) {
                const int rc = run_plain(s, r);
                if (rc)
                    r->res.status = rc;
            }
            retire(s, batch, t0);
            continue;
        }
        if (flights.empty())
            continue;
        Flight &f = flights.front();
        // with room for another run, keep polling (arrivals get planned and
        // enqueued behind it); with two in flight, wait for the oldest
        if (f.rc == SCR_OK && flights.size() < 2 && cudaEventQuery(s->slots[f.slot].done) == cudaErrorNotReady) {
            cudaGetLastError();
            continue;
        }
        cudaGetLastError();
        if (f.rc == SCR_OK)
            f.rc = finish_batched(s, s->slots[f.slot], f.reqs);
        if (f.rc)
            for (SrvRequest *r : f.reqs)
                r->res.status = f.rc;
        s->slots[f.slot].busy = false;
        retire(s, f.reqs, f.t0);
        flights.pop_front();
    }
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
    if (cfg->words_per_warp && cfg->words_per_warp != 2 && cfg->words_per_warp != 4 && cfg->words_per_warp != 8)
        return fail(SCR_EINVAL, "words_per_warp must be 0, 2, 4 or 8");
    if (cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 16 || cfg->max_batch < 0)
        return fail(SCR_EINVAL, "blocks_per_sm must be in [0, 16] and max_batch >= 0");
    *out = nullptr;
    DeviceGuard dg(c->device);
    auto *s = new (std::nothrow) scr_server();
    if (!s)
        return fail(SCR_ENOMEM, "host allocation failed");
    s->ctx = c;
    s->cfg = *cfg;
    s->hold = cfg->start_held != 0;
    // table builds go first when they and screening kernels wait for the same SMs
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    cudaError_t e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    for (auto &bd : s->builders)
        if (e == cudaSuccess)
            e = cudaStreamCreateWithPriority(&bd.st, cudaStreamNonBlocking, prio_hi);
    if (e != cudaSuccess) {
        if (s->st)
            cudaStreamDestroy(s->st);
        for (auto &bd : s->builders)
            if (bd.st)
                cudaStreamDestroy(bd.st);
        delete s;
        return fail(SCR_ECUDA, "stream creation: %s", cudaGetErrorString(e));
    }
    for (auto &sl : s->slots)
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        for (auto &sl : s->slots)
            if (sl.done)
                cudaEventDestroy(sl.done);
        cudaStreamDestroy(s->st);
        for (auto &bd : s->builders)
            cudaStreamDestroy(bd.st);
        delete s;
        return fail(SCR_ECUDA, "event creation: %s", cudaGetErrorString(e));
    }
    if (cfg->table_budget_bytes) {
        const size_t want = (size_t)cfg->table_budget_bytes + (size_t)(cfg->table_budget_bytes >> 4);
        if ((rc = dev_alloc(c, (want + kArenaAlign - 1) & ~(kArenaAlign - 1), s->st, &s->arena))) {
            cudaStreamDestroy(s->st);
            for (auto &bd : s->builders)
                cudaStreamDestroy(bd.st);
            for (auto &sl : s->slots)
                cudaEventDestroy(sl.done);
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
    for (auto &sl : s->slots)
        for (DevBuf *b : {&sl.mask_dev, &sl.segs_dev, &sl.scratch_dev})
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
    for (auto &sl : s->slots) {
        for (DevBuf *b : {&sl.desc_host, &sl.out_host})
            if (b->p)
                cudaFreeHost(b->p);
        cudaEventDestroy(sl.done);
    }
    cudaStreamDestroy(s->st);
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
