// spv_pipe.cu -- a batch held in host memory, processed chunk by chunk with
// the host->device copies, the kernels and the device->host copies of
// different chunks overlapped.
//
// A batch that starts and ends in host memory is bound by the PCIe copies,
// not by the kernels: its words go up once and its text, several times
// larger, comes back once. Chunks of whole modules rotate over `depth` slots,
// each with its own stream and device buffers, so while one chunk's text is
// copied back the next chunk's kernels run and the one after it is copied
// up. The host finishes chunk c-1 (reads its text size, places its text)
// right after queueing chunk c, so the device->host copy engine always has
// the next text queued.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/spv.h"

namespace {

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t small_done = nullptr;    // status, error rows and text offsets are back
    char *dev = nullptr;                 // one device block, carved below
    size_t dev_bytes = 0;
    char *text = nullptr;                // device text buffer
    uint64_t text_cap = 0;
    int64_t *h_off = nullptr;            // pinned: the chunk's module offsets, rebased to its first word
    uint64_t *h_toff = nullptr;          // pinned: the chunk's text offsets
    int64_t cap_words = 0;
    int32_t cap_mods = 0;
    // carved device buffers
    uint32_t *words = nullptr, *out = nullptr, *status = nullptr, *dstat = nullptr;
    int64_t *off = nullptr, *err = nullptr;
    uint64_t *toff = nullptr;
    spv_table table{};
    void *ws = nullptr, *dws = nullptr;
    size_t ws_bytes = 0, dws_bytes = 0;
    // the chunk in flight
    int32_t m_a = 0, m_b = 0;
    int64_t w_a = 0, w_b = 0;
};

void slot_free_buffers(Slot &s)
{
    if (s.dev) cudaFree(s.dev);
    if (s.text) cudaFree(s.text);
    if (s.h_off) cudaFreeHost(s.h_off);
    if (s.h_toff) cudaFreeHost(s.h_toff);
    s.dev = nullptr; s.text = nullptr; s.h_off = nullptr; s.h_toff = nullptr;
    s.dev_bytes = 0; s.text_cap = 0; s.cap_words = 0; s.cap_mods = 0;
}

// device buffers for chunks of up to cap_words words and cap_mods modules
int slot_reserve(Slot &s, int64_t cap_words, int32_t cap_mods, bool encode)
{
    if (cap_words <= s.cap_words && cap_mods <= s.cap_mods) return SPV_SUCCESS;
    cap_words = std::max(cap_words, s.cap_words);
    cap_mods = std::max(cap_mods, s.cap_mods);
    uint64_t text_cap = std::max<uint64_t>(s.text_cap, 10ull * (uint64_t)cap_words + 4096);
    slot_free_buffers(s);
    const int64_t rows = cap_words;                      // rows never exceed words
    // the default tile shape follows each chunk's mean module size; the
    // shape with the most tiles (2048 x 128) bounds the workspace of both
    spv_config small_tiles{};
    small_tiles.tile_words = 2048;
    small_tiles.threads = 128;
    const size_t ws_bytes = spv_workspace_bytes(cap_mods, cap_words, 0, &small_tiles);
    const size_t dws_bytes = spv_dis_workspace_bytes(cap_mods, cap_words, rows, 0);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = up256(o + bytes); return at; };
    const size_t o_words = take(4 * (size_t)cap_words), o_out = encode ? take(4 * (size_t)cap_words) : 0;
    const size_t o_off = take(8 * ((size_t)cap_mods + 1)), o_status = take(4 * (size_t)cap_mods);
    const size_t o_dstat = take(4 * (size_t)cap_mods), o_err = take(8 * (size_t)cap_mods);
    const size_t o_toff = take(8 * ((size_t)cap_mods + 1));
    const size_t o_op = take(2 * (size_t)rows), o_wc = take(2 * (size_t)rows), o_roff = take(8 * (size_t)rows);
    const size_t o_rt = take(4 * (size_t)rows), o_rid = take(4 * (size_t)rows), o_mod = take(4 * (size_t)rows);
    const size_t o_first = take(8 * ((size_t)cap_mods + 1)), o_nin = take(4 * (size_t)cap_mods);
    const size_t o_ws = take(ws_bytes), o_dws = take(dws_bytes);
    if (cudaMalloc((void **)&s.dev, o) != cudaSuccess) { s.dev = nullptr; return SPV_E_CUDA; }
    if (cudaMalloc((void **)&s.text, text_cap) != cudaSuccess) { s.text = nullptr; slot_free_buffers(s); return SPV_E_CUDA; }
    if (cudaMallocHost((void **)&s.h_off, 8 * ((size_t)cap_mods + 1)) != cudaSuccess ||
        cudaMallocHost((void **)&s.h_toff, 8 * ((size_t)cap_mods + 1)) != cudaSuccess) {
        slot_free_buffers(s);
        return SPV_E_CUDA;
    }
    s.dev_bytes = o;
    s.text_cap = text_cap;
    s.cap_words = cap_words;
    s.cap_mods = cap_mods;
    s.words = (uint32_t *)(s.dev + o_words);
    s.out = encode ? (uint32_t *)(s.dev + o_out) : nullptr;
    s.off = (int64_t *)(s.dev + o_off);
    s.status = (uint32_t *)(s.dev + o_status);
    s.dstat = (uint32_t *)(s.dev + o_dstat);
    s.err = (int64_t *)(s.dev + o_err);
    s.toff = (uint64_t *)(s.dev + o_toff);
    s.table.op = (uint16_t *)(s.dev + o_op);
    s.table.wc = (uint16_t *)(s.dev + o_wc);
    s.table.off = (uint64_t *)(s.dev + o_roff);
    s.table.rtype = (uint32_t *)(s.dev + o_rt);
    s.table.rid = (uint32_t *)(s.dev + o_rid);
    s.table.mod = (uint32_t *)(s.dev + o_mod);
    s.table.mod_first_row = (int64_t *)(s.dev + o_first);
    s.table.mod_n_instr = (uint32_t *)(s.dev + o_nin);
    s.table.capacity_rows = rows;
    s.ws = s.dev + o_ws; s.ws_bytes = ws_bytes;
    s.dws = s.dev + o_dws; s.dws_bytes = dws_bytes;
    return SPV_SUCCESS;
}

}  // namespace

struct spv_pipe {
    spv_pipe_cfg cfg{};
    int device = 0;
    std::vector<Slot> slots;
};

extern "C" spv_pipe *spv_pipe_create(const spv_pipe_cfg *cfg)
{
    spv_pipe *p = new spv_pipe();
    if (cfg) p->cfg = *cfg;
    if (p->cfg.chunk_words <= 0) p->cfg.chunk_words = 8ll << 20;
    if (p->cfg.depth <= 0) p->cfg.depth = 3;
    if (p->cfg.depth < 2) p->cfg.depth = 2;
    if (p->cfg.depth > 8) p->cfg.depth = 8;
    if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return nullptr; }
    p->slots.resize((size_t)p->cfg.depth);
    for (Slot &s : p->slots) {
        if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.small_done, cudaEventDisableTiming) != cudaSuccess) {
            spv_pipe_destroy(p);
            return nullptr;
        }
    }
    return p;
}

extern "C" void spv_pipe_destroy(spv_pipe *p)
{
    if (!p) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    for (Slot &s : p->slots) {
        if (s.st) cudaStreamSynchronize(s.st);
        slot_free_buffers(s);
        if (s.small_done) cudaEventDestroy(s.small_done);
        if (s.st) cudaStreamDestroy(s.st);
    }
    cudaSetDevice(prev);
    delete p;
}

extern "C" int spv_pipe_run(spv_pipe *p, const uint32_t *h_words, int64_t n_words, const int64_t *h_mod_off,
                            int32_t n_modules, uint32_t *h_status, int64_t *h_err_row, uint64_t *h_text_off,
                            char *h_text, uint64_t text_capacity, uint32_t *h_out_words, uint32_t *h_dis_status)
{
    if (!p || n_modules < 0 || n_words < 0 || !h_mod_off || !h_text_off) return SPV_E_ARG;
    if (n_modules && (!h_status || !h_err_row)) return SPV_E_ARG;
    if ((n_words && !h_words) || (text_capacity && !h_text)) return SPV_E_ARG;
    for (int32_t m = 0; m < n_modules; m++)
        if (h_mod_off[m] < 0 || h_mod_off[m + 1] < h_mod_off[m]) return SPV_E_ARG;
    if (n_modules && h_mod_off[n_modules] > n_words) return SPV_E_ARG;
    h_text_off[0] = 0;
    if (n_modules == 0) return SPV_SUCCESS;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(p->device) != cudaSuccess) return SPV_E_CUDA;
    struct DevGuard { int d; ~DevGuard() { cudaSetDevice(d); } } guard{prev};

    // chunks of whole modules, about chunk_words words each
    std::vector<std::pair<int32_t, int32_t>> chunks;
    int64_t max_words = 0;
    int32_t max_mods = 0;
    for (int32_t a = 0; a < n_modules;) {
        int32_t b = a + 1;
        while (b < n_modules && h_mod_off[b + 1] - h_mod_off[a] <= p->cfg.chunk_words) b++;
        chunks.emplace_back(a, b);
        max_words = std::max<int64_t>(max_words, h_mod_off[b] - h_mod_off[a]);
        max_mods = std::max(max_mods, b - a);
        a = b;
    }
    const bool encode = p->cfg.encode != 0;
    for (Slot &s : p->slots) {
        int rc = slot_reserve(s, std::max<int64_t>(max_words, 1), max_mods, encode);
        if (rc != SPV_SUCCESS) return rc;
    }
    spv_dis_opts opts{p->cfg.inline_names, p->cfg.header};
    const size_t nslot = p->slots.size();
    uint64_t base = 0;

    auto enqueue = [&](size_t c) -> int {
        Slot &s = p->slots[c % nslot];
        s.m_a = chunks[c].first; s.m_b = chunks[c].second;
        s.w_a = h_mod_off[s.m_a]; s.w_b = h_mod_off[s.m_b];
        const int32_t nm = s.m_b - s.m_a;
        const int64_t nw = s.w_b - s.w_a;
        for (int32_t i = 0; i <= nm; i++) s.h_off[i] = h_mod_off[s.m_a + i] - s.w_a;
        if (nw && cudaMemcpyAsync(s.words, h_words + s.w_a, 4 * (size_t)nw, cudaMemcpyHostToDevice, s.st) != cudaSuccess)
            return SPV_E_CUDA;
        if (cudaMemcpyAsync(s.off, s.h_off, 8 * ((size_t)nm + 1), cudaMemcpyHostToDevice, s.st) != cudaSuccess)
            return SPV_E_CUDA;
        spv_batch b{s.words, s.off, nm, nw};
        int rc = spv_process_batch(&b, &s.table, s.status, s.err, p->cfg.validate ? 1 : 0, s.out, 1, s.ws,
                                   s.ws_bytes, 0, nullptr, (spv_stream_t)s.st);
        if (rc != SPV_SUCCESS) return rc;
        rc = spv_disassemble_batch(&b, &s.table, &opts, s.text, s.text_cap, s.toff, s.dstat, s.dws, s.dws_bytes, 0,
                                   (spv_stream_t)s.st);
        if (rc != SPV_SUCCESS) return rc;
        if (cudaMemcpyAsync(h_status + s.m_a, s.status, 4 * (size_t)nm, cudaMemcpyDeviceToHost, s.st) != cudaSuccess ||
            cudaMemcpyAsync(h_err_row + s.m_a, s.err, 8 * (size_t)nm, cudaMemcpyDeviceToHost, s.st) != cudaSuccess ||
            cudaMemcpyAsync(s.h_toff, s.toff, 8 * ((size_t)nm + 1), cudaMemcpyDeviceToHost, s.st) != cudaSuccess)
            return SPV_E_CUDA;
        if (h_dis_status &&
            cudaMemcpyAsync(h_dis_status + s.m_a, s.dstat, 4 * (size_t)nm, cudaMemcpyDeviceToHost, s.st) != cudaSuccess)
            return SPV_E_CUDA;
        if (h_out_words && encode && nw &&
            cudaMemcpyAsync(h_out_words + s.w_a, s.out, 4 * (size_t)nw, cudaMemcpyDeviceToHost, s.st) != cudaSuccess)
            return SPV_E_CUDA;
        return cudaEventRecord(s.small_done, s.st) == cudaSuccess ? SPV_SUCCESS : SPV_E_CUDA;
    };

    // the chunk's text size is known: place its offsets and copy its text
    // (the part below text_capacity) to the running base
    auto finish = [&](size_t c) -> int {
        Slot &s = p->slots[c % nslot];
        if (cudaEventSynchronize(s.small_done) != cudaSuccess) return SPV_E_CUDA;
        const int32_t nm = s.m_b - s.m_a;
        uint64_t size = s.h_toff[nm];
        if (size > s.text_cap) {
            // the chunk's text outgrew the slot's buffer: grow it and rerun
            // the disassembly of this chunk (its table is still on the slot)
            if (cudaStreamSynchronize(s.st) != cudaSuccess) return SPV_E_CUDA;
            cudaFree(s.text);
            s.text = nullptr;
            uint64_t cap = size + size / 4 + 4096;
            if (cudaMalloc((void **)&s.text, cap) != cudaSuccess) { s.text = nullptr; s.text_cap = 0; return SPV_E_CUDA; }
            s.text_cap = cap;
            spv_batch b{s.words, s.off, nm, s.w_b - s.w_a};
            int rc = spv_disassemble_batch(&b, &s.table, &opts, s.text, s.text_cap, s.toff, s.dstat, s.dws,
                                           s.dws_bytes, 0, (spv_stream_t)s.st);
            if (rc != SPV_SUCCESS) return rc;
            if (cudaMemcpyAsync(s.h_toff, s.toff, 8 * ((size_t)nm + 1), cudaMemcpyDeviceToHost, s.st) != cudaSuccess)
                return SPV_E_CUDA;
            if (h_dis_status && cudaMemcpyAsync(h_dis_status + s.m_a, s.dstat, 4 * (size_t)nm,
                                                cudaMemcpyDeviceToHost, s.st) != cudaSuccess)
                return SPV_E_CUDA;
            if (cudaStreamSynchronize(s.st) != cudaSuccess) return SPV_E_CUDA;
            size = s.h_toff[nm];
        }
        for (int32_t i = 0; i < nm; i++) h_text_off[s.m_a + i] = base + s.h_toff[i];
        const uint64_t room = text_capacity > base ? text_capacity - base : 0;
        const uint64_t n = size < room ? size : room;
        if (n && cudaMemcpyAsync(h_text + base, s.text, n, cudaMemcpyDeviceToHost, s.st) != cudaSuccess)
            return SPV_E_CUDA;
        base += size;
        return SPV_SUCCESS;
    };

    int rc = SPV_SUCCESS;
    for (size_t c = 0; c < chunks.size() && rc == SPV_SUCCESS; c++) {
        rc = enqueue(c);
        if (rc == SPV_SUCCESS && c >= 1) rc = finish(c - 1);
    }
    if (rc == SPV_SUCCESS) rc = finish(chunks.size() - 1);
    for (Slot &s : p->slots)
        if (cudaStreamSynchronize(s.st) != cudaSuccess && rc == SPV_SUCCESS) rc = SPV_E_CUDA;
    h_text_off[n_modules] = base;
    return rc;
}
