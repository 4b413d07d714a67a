// spv_serve.cu -- continuous-batching server over the batched kernels.
//
// Modules arrive one by one (a JIT backend emitting kernels, the paper's use
// case in section 4). A scheduler thread forms a batch from every waiting
// module whenever one of NSLOT batch slots is free, and runs decode +
// validate + disassembly on it (spv_process_batch, spv_disassemble_batch) on
// that slot's stream; a small kernel then writes the batch's text straight
// into mapped pinned host memory, and one stream callback per batch wakes
// the scheduler when its kernels and copies finish. Requests that arrive while a batch is on the GPU wait
// for the next free slot. Admission is by device footprint: a module of n
// words holds 28 * n + 64 bytes of the device pool (words and decoded
// table) from submit to release.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <time.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <algorithm>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/spv.h"

namespace {

uint64_t now_ns()
{
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

size_t up(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int NSLOT = 3;                 // batches on the GPU at once

// the batch's text (text_off[n] bytes, when it fits cap) to pinned host
// memory mapped into the device's address space: 16-byte stores where the
// two buffers share a phase, bytes elsewhere
__global__ void k_text_to_host(const char *src, const uint64_t *total_at, char *dst, uint64_t cap)
{
    const uint64_t total = *total_at;
    if (total > cap) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (((((uintptr_t)src) ^ ((uintptr_t)dst)) & 15) == 0) {
        const uint64_t head = (16 - (((uintptr_t)src) & 15)) & 15;
        const uint64_t h = head < total ? head : total;
        for (uint64_t i = t0; i < h; i += stride) dst[i] = src[i];
        const uint64_t nv = (total - h) / 16;
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src + h);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst + h);
        for (uint64_t i = t0; i < nv; i += stride) d4[i] = s4[i];
        for (uint64_t i = h + 16 * nv + t0; i < total; i += stride) dst[i] = src[i];
    } else {
        for (uint64_t i = t0; i < total; i += stride) dst[i] = src[i];
    }
}

// first-fit allocator over the byte range [0, size)
class Arena {
    std::map<size_t, size_t> free_;   // offset -> length
public:
    void init(size_t n) { free_.clear(); if (n) free_[0] = n; }
    bool alloc(size_t n, size_t *off)
    {
        n = up(n ? n : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            size_t o = it->first, rest = it->second - n;
            free_.erase(it);
            if (rest) free_[o + n] = rest;
            *off = o;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = up(n ? n : 1);
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
        }
    }
};

struct Batch;

struct Region { size_t off = 0, bytes = 0; bool held = false; };

struct Req {
    uint64_t ticket = 0;
    int64_t n_words = 0;
    Region stage;                        // the module's words in the pinned pool until its batch completes
    uint64_t submit_ns = 0, done_ns = 0;
    int state = 0;                       // 0 queued, 1 in flight, 2 done
    uint64_t footprint = 0;
    Batch *batch = nullptr;
    int index = 0;
};

struct Batch {
    spv_server *srv = nullptr;
    std::vector<Req *> reqs;
    int64_t words = 0;
    int n = 0;
    int slot = 0;
    int error = SPV_SUCCESS;
    std::atomic<int> signaled{0};
    int handled = 0;
    int phase = 0;                       // 1 kernels, text and small copies; 2 text copied again (past its first room)
    int live = 0;
    Region dev, tmp, text_extra, pin_small, pin_text;
    // device pointers
    uint32_t *d_words = nullptr; int64_t *d_off = nullptr;
    uint16_t *d_op = nullptr, *d_wc = nullptr; uint64_t *d_roff = nullptr;
    uint32_t *d_rtype = nullptr, *d_rid = nullptr, *d_mod = nullptr;
    int64_t *d_first = nullptr; uint32_t *d_ninstr = nullptr;
    uint32_t *d_status = nullptr; int64_t *d_err = nullptr; uint64_t *d_toff = nullptr; uint32_t *d_dst = nullptr;
    char *d_text = nullptr; uint64_t text_cap = 0;
    void *d_ws = nullptr; size_t ws_bytes = 0; void *d_dws = nullptr; size_t dws_bytes = 0;
    // pinned host pointers
    int64_t *h_modoff = nullptr;
    uint32_t *h_status = nullptr; int64_t *h_err = nullptr; uint64_t *h_toff = nullptr;
    int64_t *h_first = nullptr; uint32_t *h_ninstr = nullptr; char *h_text = nullptr;
};

}  // namespace

struct spv_server {
    spv_serve_cfg cfg{};
    int dev = 0;
    char *dpool = nullptr;
    size_t dpool_bytes = 0;
    Arena darena;
    char *hpool = nullptr;
    size_t hpool_bytes = 0;
    Arena harena;
    char *hpool_dev = nullptr;           // the pinned pool's address on the device
    cudaStream_t st[NSLOT] = {};
    bool slot_busy[NSLOT] = {};
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, Req *> reqs;
    std::vector<Batch *> inflight;
    uint64_t next_ticket = 1;
    uint64_t committed = 0;
    bool stop = false;
    std::thread th;
};

namespace {

// the stream callback of a batch. The server is read before the batch is
// signaled: from then on the scheduler may complete the batch and its
// results may be released, freeing it while this callback still runs (a read
// of the freed batch here once blocked the driver's callback thread, and
// with it every stream of the server).
void CUDART_CB on_stage(void *p)
{
    Batch *b = (Batch *)p;
    spv_server *srv = b->srv;
    b->signaled.fetch_add(1);
    srv->cv.notify_all();
}

bool dalloc(spv_server *s, Region &r, size_t bytes)
{
    if (!s->darena.alloc(bytes, &r.off)) return false;
    r.bytes = bytes; r.held = true;
    return true;
}
bool halloc(spv_server *s, Region &r, size_t bytes)
{
    if (!s->harena.alloc(bytes, &r.off)) return false;
    r.bytes = bytes; r.held = true;
    return true;
}
void dfree(spv_server *s, Region &r) { if (r.held) { s->darena.release(r.off, r.bytes); r.held = false; } }
void hfree(spv_server *s, Region &r) { if (r.held) { s->harena.release(r.off, r.bytes); r.held = false; } }

// carve consecutive sub-buffers out of one region
struct Carver {
    char *base; size_t used = 0;
    template <class T> T *take(size_t count)
    {
        T *p = (T *)(base + used);
        used = up(used + sizeof(T) * (count ? count : 1));
        return p;
    }
};

size_t persistent_bytes(int n, int64_t w)
{
    return up(4 * (size_t)w) + up(8 * (size_t)(n + 1)) + 2 * up(2 * (size_t)w) + up(8 * (size_t)w) +
           3 * up(4 * (size_t)w) + up(8 * (size_t)(n + 1)) + up(4 * (size_t)n) + 4096;
}

void finish_requests(spv_server *s, Batch *b)
{
    uint64_t t = now_ns();
    for (Req *r : b->reqs) { r->state = 2; r->done_ns = t; }
    s->done_cv.notify_all();
}

// launch a batch on a free slot; returns false when memory is short. The
// server lock is held for the bookkeeping and released for the CUDA calls.
// The batch is the waiting modules from the front of the queue, up to the
// batch limits; when its memory does not fit (the pools are first-fit and
// fragment over a long run), it takes half as many, down to the oldest
// module alone. A batch that only grew while its memory did not fit would
// never go out: the queue keeps growing behind it.
bool launch(spv_server *s, int slot, std::unique_lock<std::mutex> &lk)
{
    size_t cnt = 0;
    int64_t words = 0;
    for (Req *r : s->queue) {
        if ((int)cnt >= s->cfg.max_batch_modules) break;
        if (cnt && words + r->n_words > s->cfg.max_batch_words) break;
        words += r->n_words;
        cnt++;
    }
    if (!cnt) return false;
    Batch *b = new Batch();
    for (;;) {
        const int n = (int)cnt;
        b->ws_bytes = spv_workspace_bytes(n, words, 0, nullptr);
        b->dws_bytes = spv_dis_workspace_bytes(n, words, words, 0);
        b->text_cap = 12ull * (uint64_t)words + 512ull * n + 1024;
        size_t tmp_bytes = up(b->ws_bytes) + up(b->dws_bytes) + up(b->text_cap) + up(4 * (size_t)n) +
                           up(8 * (size_t)n) + up(8 * (size_t)(n + 1)) + up(4 * (size_t)n) + 4096;
        size_t small = up(8 * (size_t)(n + 1)) * 3 + up(4 * (size_t)n) * 2 + up(8 * (size_t)n) + 4096;
        bool ok = dalloc(s, b->dev, persistent_bytes(n, words));
        ok = ok && dalloc(s, b->tmp, tmp_bytes);
        ok = ok && halloc(s, b->pin_small, small);
        ok = ok && halloc(s, b->pin_text, b->text_cap + 1);
        if (ok) break;
        dfree(s, b->dev); dfree(s, b->tmp); hfree(s, b->pin_small); hfree(s, b->pin_text);
        if (cnt == 1) { delete b; return false; }
        cnt = (cnt + 1) / 2;
        words = 0;
        for (size_t i = 0; i < cnt; i++) words += s->queue[i]->n_words;
    }
    std::vector<Req *> take(s->queue.begin(), s->queue.begin() + (long)cnt);
    s->queue.erase(s->queue.begin(), s->queue.begin() + (long)cnt);
    b->srv = s;
    b->reqs = take;
    b->words = words;
    b->n = (int)cnt;
    b->slot = slot;
    int n = b->n;
    Carver dv{s->dpool + b->dev.off};
    b->d_words = dv.take<uint32_t>(words);
    b->d_off = dv.take<int64_t>(n + 1);
    b->d_op = dv.take<uint16_t>(words); b->d_wc = dv.take<uint16_t>(words);
    b->d_roff = dv.take<uint64_t>(words);
    b->d_rtype = dv.take<uint32_t>(words); b->d_rid = dv.take<uint32_t>(words); b->d_mod = dv.take<uint32_t>(words);
    b->d_first = dv.take<int64_t>(n + 1); b->d_ninstr = dv.take<uint32_t>(n);
    Carver tv{s->dpool + b->tmp.off};
    b->d_ws = tv.take<char>(b->ws_bytes); b->d_dws = tv.take<char>(b->dws_bytes);
    b->d_text = tv.take<char>(b->text_cap);
    b->d_status = tv.take<uint32_t>(n); b->d_err = tv.take<int64_t>(n);
    b->d_toff = tv.take<uint64_t>(n + 1); b->d_dst = tv.take<uint32_t>(n);
    Carver hv{s->hpool + b->pin_small.off};
    b->h_modoff = hv.take<int64_t>(n + 1); b->h_toff = hv.take<uint64_t>(n + 1); b->h_first = hv.take<int64_t>(n + 1);
    b->h_status = hv.take<uint32_t>(n); b->h_ninstr = hv.take<uint32_t>(n); b->h_err = hv.take<int64_t>(n);
    b->h_text = s->hpool + b->pin_text.off;
    cudaStream_t st = s->st[slot];
    // module offsets, and the words: one copy per run of contiguous staging
    int64_t o = 0;
    for (int i = 0; i < n; i++) { b->h_modoff[i] = o; take[i]->batch = b; take[i]->index = i; take[i]->state = 1; o += take[i]->n_words; }
    b->h_modoff[n] = o;
    s->slot_busy[slot] = true;
    lk.unlock();
    int rc = cudaSuccess;
    int i = 0;
    while (i < n && rc == cudaSuccess) {
        int j = i;
        size_t bytes = 4 * (size_t)take[i]->n_words;
        // merge modules whose staged words follow each other exactly
        while (j + 1 < n && take[j + 1]->stage.off == take[j]->stage.off + up(take[j]->stage.bytes) &&
               up(take[j]->stage.bytes) == 4 * (size_t)take[j]->n_words) {
            j++;
            bytes += 4 * (size_t)take[j]->n_words;
        }
        if (bytes) rc = cudaMemcpyAsync(b->d_words + b->h_modoff[i], s->hpool + take[i]->stage.off, bytes,
                                        cudaMemcpyHostToDevice, st);
        i = j + 1;
    }
    if (rc == cudaSuccess) rc = cudaMemcpyAsync(b->d_off, b->h_modoff, 8 * (size_t)(n + 1), cudaMemcpyHostToDevice, st);
    spv_batch bt{b->d_words, b->d_off, n, words};
    spv_table tb{b->d_op, b->d_wc, b->d_roff, b->d_rtype, b->d_rid, b->d_mod, b->d_first, b->d_ninstr, words};
    int e = rc == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
    if (e == SPV_SUCCESS)
        e = spv_process_batch(&bt, &tb, b->d_status, b->d_err, 1, nullptr, 0, b->d_ws, b->ws_bytes, 0, nullptr,
                              (spv_stream_t)st);
    spv_dis_opts opts{s->cfg.inline_names, s->cfg.header};
    if (e == SPV_SUCCESS)
        e = spv_disassemble_batch(&bt, &tb, &opts, b->d_text, b->text_cap, b->d_toff, b->d_dst, b->d_dws,
                                  b->dws_bytes, 0, (spv_stream_t)st);
    if (e == SPV_SUCCESS) {
        const int blocks = (int)std::min<uint64_t>(1024, (b->text_cap / 16 + 255) / 256 + 1);
        k_text_to_host<<<blocks, 256, 0, st>>>(b->d_text, b->d_toff + n, s->hpool_dev + b->pin_text.off, b->text_cap);
        if (cudaPeekAtLastError() != cudaSuccess) e = SPV_E_CUDA;
    }
    if (e == SPV_SUCCESS) {
        cudaMemcpyAsync(b->h_status, b->d_status, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(b->h_err, b->d_err, 8 * (size_t)n, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(b->h_toff, b->d_toff, 8 * (size_t)(n + 1), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(b->h_first, b->d_first, 8 * (size_t)(n + 1), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(b->h_ninstr, b->d_ninstr, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
        if (cudaLaunchHostFunc(st, on_stage, b) != cudaSuccess) e = SPV_E_CUDA;
    }
    lk.lock();
    b->phase = 1;
    s->inflight.push_back(b);
    if (e != SPV_SUCCESS) {
        b->error = e;
        b->signaled.store(99);
    }
    return true;
}

// the batch's stream has finished everything it launched: free the
// transient device memory and the staged words, publish the results
void complete(spv_server *s, Batch *b)
{
    // after an error, work launched for the batch may still be running
    if (b->error != SPV_SUCCESS) cudaStreamSynchronize(s->st[b->slot]);
    dfree(s, b->tmp);
    dfree(s, b->text_extra);
    s->slot_busy[b->slot] = false;
    for (Req *r : b->reqs) hfree(s, r->stage);
    finish_requests(s, b);
    b->live = b->n;
}

// advance a batch whose stream reached its callback
void advance(spv_server *s, Batch *b)
{
    cudaStream_t st = s->st[b->slot];
    if (b->error != SPV_SUCCESS) { complete(s, b); return; }
    if (b->phase == 1) {
        uint64_t total = b->h_toff[b->n];
        if (total > b->text_cap && !b->text_extra.held) {
            // the text did not fit: disassemble again into a buffer of the
            // exact size (freed with the batch's transient memory)
            if (!dalloc(s, b->text_extra, total + 256)) { b->error = SPV_E_BUSY; complete(s, b); return; }
            b->d_text = s->dpool + b->text_extra.off;
            b->text_cap = total;
            spv_batch bt{b->d_words, b->d_off, b->n, b->words};
            spv_table tb{b->d_op, b->d_wc, b->d_roff, b->d_rtype, b->d_rid, b->d_mod, b->d_first, b->d_ninstr, b->words};
            spv_dis_opts opts{s->cfg.inline_names, s->cfg.header};
            int e = spv_disassemble_batch(&bt, &tb, &opts, b->d_text, b->text_cap, b->d_toff, b->d_dst, b->d_dws,
                                          b->dws_bytes, 0, (spv_stream_t)st);
            if (e != SPV_SUCCESS) { b->error = e; complete(s, b); return; }
            cudaMemcpyAsync(b->h_toff, b->d_toff, 8 * (size_t)(b->n + 1), cudaMemcpyDeviceToHost, st);
            if (cudaLaunchHostFunc(st, on_stage, b) != cudaSuccess) { b->error = SPV_E_CUDA; complete(s, b); }
            return;                     // phase 1 again, now with room for the text
        }
        if (total + 1 > b->pin_text.bytes) {
            // the text outgrew its first room: copy it into a pinned region of its size
            hfree(s, b->pin_text);
            if (!halloc(s, b->pin_text, total + 1)) { b->error = SPV_E_BUSY; complete(s, b); return; }
            b->h_text = s->hpool + b->pin_text.off;
            if (total) cudaMemcpyAsync(b->h_text, b->d_text, total, cudaMemcpyDeviceToHost, st);
            b->phase = 2;
            if (cudaLaunchHostFunc(st, on_stage, b) != cudaSuccess) { b->error = SPV_E_CUDA; complete(s, b); }
            return;
        }
        // the text is in pinned memory already (written by k_text_to_host)
    }
    complete(s, b);
}

void scheduler(spv_server *s)
{
    cudaSetDevice(s->dev);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        for (size_t k = 0; k < s->inflight.size();) {
            Batch *b = s->inflight[k];
            int sig = b->signaled.load();
            if (sig == 99 || sig > b->handled) {
                if (sig != 99) b->handled = sig;
                else b->signaled.store(b->handled);
                advance(s, b);
                bool done = b->reqs.empty() || b->reqs[0]->state == 2;
                if (done) { s->inflight.erase(s->inflight.begin() + k); continue; }
            }
            k++;
        }
        // stopping: the batches in flight finish, queued modules are dropped
        if (s->stop && s->inflight.empty()) break;
        bool launched = false;
        for (int slot = 0; slot < NSLOT && !s->stop && !s->queue.empty(); slot++)
            if (!s->slot_busy[slot]) launched |= launch(s, slot, lk);
        if (!launched) s->cv.wait_for(lk, std::chrono::microseconds(50));
    }
}

void fill(const spv_server *s, const Req *r, spv_result *out)
{
    const Batch *b = r->batch;
    memset(out, 0, sizeof(*out));
    out->submit_ns = r->submit_ns;
    out->done_ns = r->done_ns;
    if (!b) return;
    out->error = b->error;
    out->batch_modules = (uint32_t)b->n;
    if (b->error != SPV_SUCCESS) return;
    int i = r->index;
    out->status = b->h_status[i];
    out->err_row = b->h_err[i];
    out->n_instr = b->h_ninstr[i];
    out->text = b->h_text ? b->h_text + b->h_toff[i] : nullptr;
    out->text_len = b->h_toff[i + 1] - b->h_toff[i];
    int64_t f = b->h_first[i];
    out->op = b->d_op + f; out->wc = b->d_wc + f; out->rtype = b->d_rtype + f; out->rid = b->d_rid + f;
    out->off = b->d_roff + f;
    out->words_base = b->d_words;
}

}  // namespace

extern "C" spv_server *spv_serve_create(const spv_serve_cfg *cfg)
{
    spv_server *s = new spv_server();
    if (cfg) s->cfg = *cfg;
    if (!s->cfg.hbm_cap_bytes) s->cfg.hbm_cap_bytes = 8ull << 30;
    if (s->cfg.max_batch_words <= 0) s->cfg.max_batch_words = 32ll << 20;
    if (s->cfg.max_batch_modules <= 0) s->cfg.max_batch_modules = 4096;
    s->dev = s->cfg.device;
    if (cudaSetDevice(s->dev) != cudaSuccess) { delete s; return nullptr; }
    int64_t W = s->cfg.max_batch_words;
    spv_config small_tiles{};                      // the default shape with the most tiles bounds the workspace
    small_tiles.tile_words = 2048;
    small_tiles.threads = 128;
    size_t per_batch = spv_workspace_bytes(s->cfg.max_batch_modules, W, 0, &small_tiles) +
                       spv_dis_workspace_bytes(s->cfg.max_batch_modules, W, W, 0) + 12ull * W + 64ull * 4096 +
                       64ull * s->cfg.max_batch_modules + (1 << 20);
    s->dpool_bytes = s->cfg.hbm_cap_bytes + NSLOT * per_batch + 28ull * W;
    s->hpool_bytes = s->cfg.hbm_cap_bytes / 2 + (64ull << 20);
    if (cudaMalloc((void **)&s->dpool, s->dpool_bytes) != cudaSuccess) { delete s; return nullptr; }
    if (cudaHostAlloc((void **)&s->hpool, s->hpool_bytes, cudaHostAllocMapped) != cudaSuccess) {
        cudaFree(s->dpool); delete s; return nullptr;
    }
    if (cudaHostGetDevicePointer((void **)&s->hpool_dev, s->hpool, 0) != cudaSuccess) {
        cudaFree(s->dpool); cudaFreeHost(s->hpool); delete s; return nullptr;
    }
    s->darena.init(s->dpool_bytes);
    s->harena.init(s->hpool_bytes);
    for (int k = 0; k < NSLOT; k++) cudaStreamCreateWithFlags(&s->st[k], cudaStreamNonBlocking);
    s->th = std::thread(scheduler, s);
    return s;
}

extern "C" int spv_serve_submit(spv_server *s, const uint32_t *host_words, int64_t n_words, uint64_t *ticket)
{
    if (!s || !ticket || n_words < 0 || (n_words && !host_words)) return SPV_E_ARG;
    uint64_t fp = 28ull * (uint64_t)n_words + 64;
    const uint64_t t_submit = now_ns();
    Req *r = nullptr;
    {
        // admission and the staging region under the lock; the copy into it
        // outside, so that the scheduler is not held up by it
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return SPV_E_ARG;
        if (s->committed + fp > s->cfg.hbm_cap_bytes) return SPV_E_BUSY;
        r = new Req();
        r->n_words = n_words;
        if (!halloc(s, r->stage, 4 * (size_t)n_words)) { delete r; return SPV_E_BUSY; }
        r->footprint = fp;
        s->committed += fp;
    }
    if (n_words) memcpy(s->hpool + r->stage.off, host_words, 4 * (size_t)n_words);
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    r->submit_ns = t_submit;
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
    s->cv.notify_all();
    return SPV_SUCCESS;
}

extern "C" int spv_serve_poll(spv_server *s, uint64_t ticket, spv_result *out)
{
    if (!s || !out) return SPV_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return SPV_E_ARG;
    if (it->second->state != 2) return 0;
    fill(s, it->second, out);
    return 1;
}

extern "C" int spv_serve_wait(spv_server *s, uint64_t ticket, spv_result *out, int64_t timeout_us)
{
    if (!s || !out || timeout_us < 0) return SPV_E_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return SPV_E_ARG;
    Req *r = it->second;
    s->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->state == 2; });
    if (r->state != 2) return 0;
    fill(s, r, out);
    return 1;
}

extern "C" int spv_serve_release(spv_server *s, uint64_t ticket)
{
    if (!s) return SPV_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second->state != 2) return SPV_E_ARG;
    Req *r = it->second;
    s->reqs.erase(it);
    s->committed -= r->footprint;
    Batch *b = r->batch;
    delete r;
    if (b && --b->live <= 0) {
        dfree(s, b->dev);
        hfree(s, b->pin_small);
        hfree(s, b->pin_text);
        delete b;
    }
    return SPV_SUCCESS;
}

extern "C" void spv_serve_destroy(spv_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    for (int k = 0; k < NSLOT; k++) if (s->st[k]) { cudaStreamSynchronize(s->st[k]); cudaStreamDestroy(s->st[k]); }
    std::vector<Batch *> batches;
    for (auto &kv : s->reqs) {
        Batch *b = kv.second->batch;
        if (b && std::find(batches.begin(), batches.end(), b) == batches.end()) batches.push_back(b);
        delete kv.second;
    }
    for (Batch *b : batches) delete b;
    cudaFree(s->dpool);
    cudaFreeHost(s->hpool);
    delete s;
}

// Load replay: modules submitted at scheduled times from a native thread,
// collected in order by the calling thread. Measures the server under a
// given arrival process without the caller's own submission costs in the
// way.
extern "C" int spv_serve_replay(spv_server *s, int32_t n, const uint32_t *const *mods, const int64_t *n_words,
                                const int64_t *arrive_ns, int64_t *latency_ns, int64_t *server_ns,
                                uint32_t *batch_modules, int64_t *busy_retries)
{
    if (!s || n < 0 || (n && (!mods || !n_words || !arrive_ns || !latency_ns))) return SPV_E_ARG;
    for (int32_t i = 0; i < n; i++)
        if (arrive_ns[i] < 0 || (i && arrive_ns[i] < arrive_ns[i - 1]) || n_words[i] < 0) return SPV_E_ARG;
    std::vector<uint64_t> tickets((size_t)n);
    std::atomic<int32_t> submitted{0};
    std::atomic<int> failed{0};
    std::atomic<int64_t> busy{0};
    std::atomic<bool> stop{false};                   // the collector gave up: submit no more
    const uint64_t t0 = now_ns() + 1000000;         // start 1 ms from now
    std::thread sub([&] {
        for (int32_t i = 0; i < n && !stop.load(std::memory_order_relaxed); i++) {
            const uint64_t target = t0 + (uint64_t)arrive_ns[i];
            for (;;) {
                const uint64_t now = now_ns();
                if (now >= target) break;
                if (target - now > 200000) std::this_thread::sleep_for(std::chrono::nanoseconds(target - now - 100000));
            }
            for (;;) {
                const int rc = spv_serve_submit(s, mods[i], n_words[i], &tickets[(size_t)i]);
                if (rc == SPV_SUCCESS) break;
                if (rc != SPV_E_BUSY) { failed.store(rc); submitted.store(n + 1, std::memory_order_release); return; }
                if (stop.load(std::memory_order_relaxed)) return;
                busy.fetch_add(1);
                std::this_thread::sleep_for(std::chrono::microseconds(10));
            }
            submitted.store(i + 1, std::memory_order_release);
        }
    });
    int rc = SPV_SUCCESS;
    for (int32_t i = 0; i < n && rc == SPV_SUCCESS; i++) {
        int32_t got;
        while ((got = submitted.load(std::memory_order_acquire)) <= i) std::this_thread::yield();
        if (got > n) { rc = failed.load(); break; }
        spv_result r{};
        const int w = spv_serve_wait(s, tickets[(size_t)i], &r, 60000000);
        if (w != 1) { rc = w < 0 ? w : SPV_E_CUDA; break; }
        latency_ns[i] = (int64_t)(r.done_ns - (t0 + (uint64_t)arrive_ns[i]));
        if (server_ns) server_ns[i] = (int64_t)(r.done_ns - r.submit_ns);
        if (batch_modules) batch_modules[i] = r.batch_modules;
        spv_serve_release(s, tickets[(size_t)i]);
    }
    if (rc != SPV_SUCCESS) stop.store(true, std::memory_order_relaxed);
    sub.join();
    if (busy_retries) *busy_retries = busy.load();
    return rc;
}
