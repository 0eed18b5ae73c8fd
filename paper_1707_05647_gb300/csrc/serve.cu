// Serving loop of include/screen.h: one worker thread per server takes every
// queued request whenever it is free (continuous batching), keeps the tables of
// the images it needs resident under a table budget (least recently used
// unpinned tables are evicted; evicted tables are rebuilt from the host copy),
// screens the batch's screen requests in one batched run or one plain launch
// pair each, and writes each request's list in compact_mask's format.
#include <condition_variable>
#include <deque>
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

struct SrvImage {
    int64_t id = 0;
    const uint8_t *host = nullptr;   // pixels (own copy or borrowed)
    std::vector<uint8_t> own;
    int H = 0, W = 0;
    int64_t pitch = 0;
    scr_tables *t = nullptr;         // resident tables, or null
    uint64_t last_use = 0;           // LRU stamp (worker only)
    int builds = 0;                  // worker only
    // under the server lock: queued or running requests naming the image, and
    // whether server_forget dropped it (freed once no request names it)
    int refs = 0;
    bool forgotten = false;
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
    std::condition_variable cv_work, cv_done;
    std::deque<SrvRequest *> pending;
    std::unordered_map<uint64_t, SrvRequest *> reqs;   // submitted, not yet collected
    std::unordered_map<int64_t, SrvImage *> images;
    std::vector<SrvImage *> dropped;                   // forgotten, tables still to free (worker)
    uint64_t next_req = 1;
    int64_t next_image = 1;
    bool stop = false, hold = false;
    std::thread worker;
    cudaStream_t st = nullptr;
    // worker state
    uint64_t lru_clock = 0, resident = 0, batch_seq = 0;
    scr_server_stats stats = {};
    DevBuf img_dev, counts_dev, keys_dev, mask_dev, list_dev, small_dev;
    DevBuf counts_host, keys_host, small_host;   // pinned
    uint64_t keys_cap = 0, list_dev_cap = 0;
};

namespace {

int grow_dev(scr_server *s, DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes)
        return SCR_OK;
    if (b.p) {
        cudaStreamSynchronize(s->st);
        dev_free(s->ctx, b.p, b.bytes, s->st);
        b.p = nullptr;
        b.bytes = 0;
    }
    bytes = std::max<size_t>(bytes, 4096);
    int rc = dev_alloc(s->ctx, bytes, s->st, &b.p);
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

uint64_t table_bytes_for(const scr_server *s, const SrvImage *im) {
    return tables_bytes(im->H, im->W, s->cfg.sum_bits, s->cfg.sq_bits);
}

void drop_tables(scr_server *s, SrvImage *im) {
    if (!im->t)
        return;
    s->resident -= im->t->bytes;
    {
        std::lock_guard<std::mutex> lk(s->ctx->mu);
        im->t->stream = s->st;
        free_tables(s->ctx, im->t);
    }
    im->t = nullptr;
}

// Make im's tables resident; images in `pinned` are not evicted.
int make_resident(scr_server *s, SrvImage *im, const std::vector<SrvImage *> &pinned, bool *built) {
    *built = false;
    if (im->t) {
        im->last_use = ++s->lru_clock;
        return SCR_OK;
    }
    const uint64_t need = table_bytes_for(s, im);
    if (s->cfg.table_budget_bytes && s->resident + need > s->cfg.table_budget_bytes) {
        std::vector<SrvImage *> cand;
        std::vector<uint64_t> bytes, last;
        std::vector<int32_t> pin;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (auto &kv : s->images)
                if (kv.second->t) {
                    cand.push_back(kv.second);
                    bytes.push_back(kv.second->t->bytes);
                    last.push_back(kv.second->last_use);
                    pin.push_back(std::find(pinned.begin(), pinned.end(), kv.second) != pinned.end());
                }
        }
        std::vector<int32_t> victims(cand.size() + 1);
        int32_t nv = 0;
        int rc = server_lru_victims(bytes.data(), last.data(), pin.data(), (int32_t)cand.size(), s->resident,
                                    s->cfg.table_budget_bytes, need, victims.data(), &nv);
        if (rc)
            return fail(SCR_EBUDGET, "image %lld: its tables (%llu bytes) do not fit the table budget",
                        (long long)im->id, (unsigned long long)need);
        for (int k = 0; k < nv; ++k) {
            drop_tables(s, cand[victims[k]]);
            s->stats.evictions++;
        }
    }
    int rc;
    if ((rc = grow_dev(s, s->img_dev, (size_t)im->H * im->W)))
        return rc;
    CUDA_TRY(cudaMemcpy2DAsync(s->img_dev.p, im->W, im->host, im->pitch, im->W, im->H, cudaMemcpyHostToDevice, s->st));
    scr_tables *t = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->ctx->mu);
        if ((rc = alloc_tables(s->ctx, im->H, im->W, s->cfg.sum_bits, s->cfg.sq_bits, s->st, &t)))
            return rc;
        if ((rc = run_build(s->ctx, (const uint8_t *)s->img_dev.p, im->H, im->W, im->W, t, s->st))) {
            free_tables(s->ctx, t);
            return rc;
        }
    }
    im->t = t;
    s->resident += t->bytes;
    s->stats.peak_resident_bytes = std::max<uint64_t>(s->stats.peak_resident_bytes, s->resident);
    im->last_use = ++s->lru_clock;
    if (im->builds++)
        s->stats.rebuilds++;
    s->stats.builds++;
    *built = true;
    return SCR_OK;
}

void deliver(SrvRequest *r, const uint64_t *keys, uint64_t count) {
    r->res.count = count;
    const uint64_t k = std::min(count, r->list_cap);
    if (k && r->list_host)
        memcpy(r->list_host, keys, k * 8);
    r->res.status = count > r->list_cap ? SCR_EOVERFLOW : SCR_OK;
}

// All screens of the batch in one batched run.
int run_batched(scr_server *s, const std::vector<SrvRequest *> &scr) {
    const int n = (int)scr.size();
    std::vector<const scr_tables *> tabs;
    std::unordered_map<SrvImage *, int> idx;
    std::vector<scr_pair> pairs(n);
    std::vector<const scr_tmpl *> tms(n);
    std::vector<scr_params> ps(n);
    for (int k = 0; k < n; ++k) {
        auto it = idx.find(scr[k]->img);
        if (it == idx.end()) {
            it = idx.emplace(scr[k]->img, (int)tabs.size()).first;
            tabs.push_back(scr[k]->img->t);
        }
        pairs[k].image = it->second;
        pairs[k].tmpl = k;
        tms[k] = scr[k]->tm;
        ps[k] = scr[k]->p;
    }
    int rc;
    if ((rc = grow_dev(s, s->counts_dev, (size_t)n * 16)) || (rc = grow_dev(s, s->small_dev, 64)) ||
        (rc = grow_host(s->counts_host, (size_t)n * 8)) || (rc = grow_host(s->small_host, 64)))
        return rc;
    if (!s->keys_cap) {
        if ((rc = grow_dev(s, s->keys_dev, (size_t)8 << 20)))
            return rc;
        s->keys_cap = s->keys_dev.bytes / 8;
    }
    uint64_t *counts = (uint64_t *)s->counts_dev.p, *offsets = counts + n;
    uint64_t *nk = (uint64_t *)s->small_dev.p, *nk_host = (uint64_t *)s->small_host.p;
    const int wpw = s->cfg.words_per_warp ? s->cfg.words_per_warp : 4;
    const int bps = s->cfg.blocks_per_sm ? s->cfg.blocks_per_sm : 4;
    for (int attempt = 0;; ++attempt) {
        scr_batch *b = nullptr;
        {
            std::lock_guard<std::mutex> lk(s->ctx->mu);
            rc = batch_prepare(s->ctx, tabs.data(), (int)tabs.size(), tms.data(), ps.data(), n, pairs.data(), n,
                               counts, offsets, nullptr, (uint64_t *)s->keys_dev.p, s->keys_cap, nk, s->st, &b);
        }
        if (rc)
            return rc;
        batch_set_shape(b, wpw, bps);
        uint64_t launches = 0;
        if (!(rc = upload_plan(b, s->st)) && !(rc = enqueue_run(b, s->st, &launches))) {
            cudaError_t e = launch_keys_to_lists((uint64_t *)s->keys_dev.p, nk, s->keys_cap, sm_count(s->ctx->device) * 4,
                                                 s->st, &launches);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(nk_host, nk, 16, cudaMemcpyDeviceToHost, s->st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s->counts_host.p, counts, (size_t)n * 8, cudaMemcpyDeviceToHost, s->st);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(s->st);
            if (e != cudaSuccess)
                rc = fail(SCR_ECUDA, "batched run: %s", cudaGetErrorString(e));
        }
        s->stats.launches += launches;
        s->ctx->launches += launches;
        {
            std::lock_guard<std::mutex> lk(s->ctx->mu);
            free_batch(s->ctx, b);
        }
        if (rc)
            return rc;
        if (nk_host[1] <= s->keys_cap)
            break;
        if (attempt)
            return fail(SCR_ECUDA, "internal: key slots grew on the repeated run");
        // the list did not fit: grow the key buffer and run the batch again
        const uint64_t want = ((nk_host[1] >> 20) + 2) << 20;
        if ((rc = grow_dev(s, s->keys_dev, want * 8)))
            return rc;
        s->keys_cap = s->keys_dev.bytes / 8;
    }
    s->stats.keys_capacity = s->keys_cap;
    const uint64_t total = nk_host[0];
    if ((rc = grow_host(s->keys_host, (size_t)std::max<uint64_t>(total, 1) * 8)))
        return rc;
    if (total) {
        CUDA_TRY(cudaMemcpyAsync(s->keys_host.p, s->keys_dev.p, total * 8, cudaMemcpyDeviceToHost, s->st));
        CUDA_TRY(cudaStreamSynchronize(s->st));
    }
    const uint64_t *cnt = (const uint64_t *)s->counts_host.p;
    const uint64_t *keys = (const uint64_t *)s->keys_host.p;
    uint64_t off = 0;
    for (int k = 0; k < n; ++k) {
        deliver(scr[k], keys + off, cnt[k]);
        off += cnt[k];
    }
    return SCR_OK;
}

// One screen with the plain single-image launches.
int run_plain(scr_server *s, SrvRequest *r) {
    const SrvImage *im = r->img;
    const int S = r->p.n_scales;
    const uint64_t words = (uint64_t)S * im->H * ((im->W + 31) / 32);
    int rc;
    if ((rc = grow_dev(s, s->mask_dev, words * 4)) || (rc = grow_dev(s, s->small_dev, 64)) ||
        (rc = grow_host(s->small_host, 64)))
        return rc;
    if (!s->list_dev_cap) {
        if ((rc = grow_dev(s, s->list_dev, (size_t)8 << 20)))
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
        if ((rc = grow_dev(s, s->list_dev, (size_t)(((want >> 20) + 1) << 20) * 8)))
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

void serve_batch(scr_server *s, std::vector<SrvRequest *> &batch) {
    const int64_t t0 = now_ns();
    const uint64_t seq = ++s->batch_seq;
    s->stats.batches++;
    std::vector<SrvImage *> dropped;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        dropped.swap(s->dropped);
    }
    for (SrvImage *im : dropped) {
        drop_tables(s, im);
        delete im;
    }
    for (SrvRequest *r : batch) {
        r->res.start_ns = t0;
        r->res.batch = seq;
        r->res.batch_size = (int32_t)batch.size();
    }
    // the images this batch uses stay resident until it ends
    std::vector<SrvImage *> pinned;
    std::vector<SrvRequest *> screens;
    for (SrvRequest *r : batch) {
        bool forgotten;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            forgotten = r->img->forgotten;
        }
        if (forgotten) {
            r->res.status = SCR_EEVICTED;
            continue;
        }
        if (r->kind == kEvict) {
            if (r->img->t && std::find(pinned.begin(), pinned.end(), r->img) == pinned.end()) {
                drop_tables(s, r->img);
                s->stats.evictions++;
            }
            r->res.status = SCR_OK;
            continue;
        }
        bool built = false;
        const int rc = make_resident(s, r->img, pinned, &built);
        r->res.built = built;
        if (rc) {
            r->res.status = rc;
            continue;
        }
        if (std::find(pinned.begin(), pinned.end(), r->img) == pinned.end())
            pinned.push_back(r->img);
        if (r->kind == kUpload)
            r->res.status = SCR_OK;
        else
            screens.push_back(r);
    }
    if (!screens.empty()) {
        if (s->cfg.mode == SCR_SERVE_BATCHED) {
            const int rc = run_batched(s, screens);
            if (rc)
                for (SrvRequest *r : screens)
                    r->res.status = rc;
        } else {
            for (SrvRequest *r : screens) {
                const int rc = run_plain(s, r);
                if (rc)
                    r->res.status = rc;
            }
        }
    }
    const int64_t t1 = now_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    for (SrvRequest *r : batch) {
        r->res.done_ns = t1;
        r->done = true;
        if (--r->img->refs == 0 && r->img->forgotten)
            s->dropped.push_back(r->img);
    }
    s->stats.resident_bytes = s->resident;
    uint64_t ri = 0;
    for (auto &kv : s->images)
        ri += kv.second->t != nullptr;
    s->stats.resident_images = ri;
    s->cv_done.notify_all();
}

void worker_main(scr_server *s) {
    cudaSetDevice(s->ctx->device);
    for (;;) {
        std::vector<SrvRequest *> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || (!s->hold && !s->pending.empty()); });
            if (s->pending.empty())
                break;   // stopping, nothing left
            const size_t lim = s->cfg.max_batch > 0 ? (size_t)s->cfg.max_batch : s->pending.size();
            while (!s->pending.empty() && batch.size() < lim) {
                batch.push_back(s->pending.front());
                s->pending.pop_front();
            }
        }
        serve_batch(s, batch);
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
    s->pending.push_back(r);
    s->stats.requests++;
    if (request_id)
        *request_id = r->id;
    s->cv_work.notify_one();
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
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return last_use[a] < last_use[b]; });
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
    cudaError_t e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete s;
        return fail(SCR_ECUDA, "stream creation: %s", cudaGetErrorString(e));
    }
    s->worker = std::thread(worker_main, s);
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
    if (im->refs == 0)
        s->dropped.push_back(im);   // the worker frees it before its next batch
    s->cv_work.notify_one();
    return SCR_OK;
}

int server_wait(scr_server *s, uint64_t request_id, int64_t timeout_us, scr_request_result *out) {
    if (!s || !out)
        return fail(SCR_EINVAL, "null server or result");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end() || request_id == 0)
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

int server_hold(scr_server *s, int32_t hold) {
    if (!s)
        return fail(SCR_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    s->hold = hold != 0;
    s->cv_work.notify_one();
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
        s->cv_work.notify_all();
    }
    if (s->worker.joinable())
        s->worker.join();
    scr_ctx *c = s->ctx;
    DeviceGuard dg(c->device);
    cudaStreamSynchronize(s->st);
    for (auto &kv : s->images) {
        drop_tables(s, kv.second);
        delete kv.second;
    }
    for (SrvImage *im : s->dropped) {
        drop_tables(s, im);
        delete im;
    }
    for (auto &kv : s->reqs)
        delete kv.second;
    for (DevBuf *b : {&s->img_dev, &s->counts_dev, &s->keys_dev, &s->mask_dev, &s->list_dev, &s->small_dev})
        dev_free(c, b->p, b->bytes, s->st);
    cudaStreamSynchronize(s->st);
    for (DevBuf *b : {&s->counts_host, &s->keys_host, &s->small_host})
        if (b->p)
            cudaFreeHost(b->p);
    cudaStreamDestroy(s->st);
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->servers.erase(s);
    }
    delete s;
}

}  // extern "C"
