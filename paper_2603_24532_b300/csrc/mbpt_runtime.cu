// libmbpt runtime: context, device arena, batch work table, the VEGAS iteration
// kernels (sample evaluation + per-chunk sums and histograms; fixed-order
// reduction, iteration combination and grid refinement) and the C ABI.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "mbpt_kernels.cuh"
#include "mbpt_kernels.h"
#include "mbpt_internal.h"

using namespace mbpt;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CUDA_TRY(expr)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(MBPT_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));         \
    } while (0)

// ---------------------------------------------------------------------------
// Device arena: first-fit allocator with coalescing over one device buffer.
// ---------------------------------------------------------------------------
struct Arena {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_blocks;   // offset -> size
    std::map<size_t, size_t> used;          // offset -> size
    static constexpr size_t kAlign = 256;

    void init(char* b, size_t s) {
        base = b;
        size = s & ~(kAlign - 1);
        free_blocks.clear();
        used.clear();
        if (size) free_blocks[0] = size;
    }
    void* alloc(size_t bytes) {
        bytes = (bytes + kAlign - 1) & ~(kAlign - 1);
        if (bytes == 0) bytes = kAlign;
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second >= bytes) {
                size_t off = it->first, sz = it->second;
                free_blocks.erase(it);
                if (sz > bytes) free_blocks[off + bytes] = sz - bytes;
                used[off] = bytes;
                return base + off;
            }
        }
        return nullptr;
    }
    void release(void* p) {
        if (!p) return;
        size_t off = (size_t)((char*)p - base);
        auto it = used.find(off);
        if (it == used.end()) return;
        size_t sz = it->second;
        used.erase(it);
        auto nx = free_blocks.lower_bound(off);
        if (nx != free_blocks.end() && off + sz == nx->first) {
            sz += nx->second;
            nx = free_blocks.erase(nx);
        }
        if (nx != free_blocks.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += sz;
                return;
            }
        }
        free_blocks[off] = sz;
    }
    size_t in_use() const {
        size_t s = 0;
        for (auto& kv : used) s += kv.second;
        return s;
    }
    size_t largest_free() const {
        size_t s = 0;
        for (auto& kv : free_blocks) s = std::max(s, kv.second);
        return s;
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// Context and integral objects
// ---------------------------------------------------------------------------
namespace {
typedef void (*IterateFn)(WorkHeader*, const WorkItem*, double*, float*);
// one k_iterate kernel per batch part (kParts: regulator, group and sixth-order bits); the shared-memory
// layout depends on the regulator and group bits only
struct KernelVariant {
    int tpb, minb;
    IterateFn fn[kParts];
    size_t smem[kParts];
};
#define MBPT_SMEM4(NW) sizeof(ChunkSmemT<NW, 0>), sizeof(ChunkSmemT<NW, 1>), sizeof(ChunkSmemT<NW, 2>), sizeof(ChunkSmemT<NW, 3>)
#define MBPT_SMEM(NW) {MBPT_SMEM4(NW), MBPT_SMEM4(NW)}
const KernelVariant kVariants[] = {
    {256, 2, {MBPT_K_ITERATE_PARTS(256, 2)}, MBPT_SMEM(8)},
    {128, 4, {MBPT_K_ITERATE_PARTS(128, 4)}, MBPT_SMEM(4)},
    {256, 1, {MBPT_K_ITERATE_PARTS(256, 1)}, MBPT_SMEM(8)},
    {128, 3, {MBPT_K_ITERATE_PARTS(128, 3)}, MBPT_SMEM(4)},
};
#undef MBPT_SMEM
#undef MBPT_SMEM4
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
}  // namespace

struct mbpt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool own_arena = false;
    Arena arena;
    int sms = 0;
    int variant = 0;                       // index into kVariants
    int variant_blocks[kNumVariants][kParts] = {};   // persistent grid of each k_iterate variant and part
    int finalize_blocks = 0;
    int spt[MBPT_MAX_DEVICE_ORDER + 1] = {};  // samples per thread of a chunk by order (kDefaultSpt at creation)
    int hist_layout = kHistWarpF32;          // per-chunk histogram layout of k_iterate
    int spin_sum = MBPT_SPIN_TABLE;          // Goldstone-sum strategy of the mixed modes
    // batch buffers (arena)
    WorkHeader* d_hdr = nullptr;
    WorkItem* d_items = nullptr;
    double** d_last_hist = nullptr;
    double* d_csum = nullptr;
    float* d_chist = nullptr;
    size_t items_cap = 0, chunks_cap = 0, hist_cap = 0;
    cudaGraphExec_t graph = nullptr;
    unsigned graph_parts = 0;              // parts whose k_iterate kernel the captured graph launches
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};   // around k_iterate and k_finalize (graph nodes)
    std::set<mbpt_diag*> diags;
    std::vector<WorkItem> h_items;
    std::vector<double*> h_last_hist;
    // batched estimate: state pointers and gathered state heads on the device (arena), and their pinned
    // host staging (gather_cap pointers, then gather_cap heads)
    const DiagState** d_gather_src = nullptr;
    uint4* d_gather_out = nullptr;
    void* h_gather = nullptr;
    size_t gather_cap = 0;
};

struct mbpt_diag {
    mbpt_ctx* ctx = nullptr;
    mbpt_diagram_desc desc;
    mbpt_physics phys;
    mbpt_vegas_cfg cfg;
    DiagRec* d_rec = nullptr;
    DiagState* d_state = nullptr;
    double* d_grid = nullptr;
    double* d_last_hist = nullptr;
    int d = 0, nb = 0;
    int n_members = 1;        // > 1: group integral, d_rec holds n_members records
    void* d_hf = nullptr;     // Hartree-Fock spectrum table (FP64 then FP32 coefficients), or null
};

namespace {

size_t state_block_bytes(int d, int nb, int n_members = 1) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return up(sizeof(DiagRec) * (size_t)n_members) + up(sizeof(DiagState)) + up(sizeof(double) * d * (nb + 1)) +
           up(sizeof(double) * d * nb);
}

void invalidate_graph(mbpt_ctx* c) {
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
}

int ensure_batch_buffers(mbpt_ctx* c, size_t n_items, size_t n_chunks, size_t hist_floats) {
    bool changed = false;
    if (!c->d_hdr) {
        c->d_hdr = (WorkHeader*)c->arena.alloc(sizeof(WorkHeader));
        if (!c->d_hdr) return fail(MBPT_ENOMEM, "arena exhausted (work header)");
        changed = true;
    }
    if (n_items > c->items_cap) {
        size_t cap = std::max(n_items, c->items_cap * 2);
        c->arena.release(c->d_items);
        c->arena.release(c->d_last_hist);
        c->d_items = (WorkItem*)c->arena.alloc(sizeof(WorkItem) * cap);
        c->d_last_hist = (double**)c->arena.alloc(sizeof(double*) * cap);
        if (!c->d_items || !c->d_last_hist) {
            c->items_cap = 0;
            return fail(MBPT_ENOMEM, "arena exhausted (work table)");
        }
        c->items_cap = cap;
        changed = true;
    }
    if (n_chunks > c->chunks_cap) {
        size_t cap = std::max(n_chunks, c->chunks_cap + c->chunks_cap / 2);
        c->arena.release(c->d_csum);
        c->d_csum = (double*)c->arena.alloc(sizeof(double) * kSumStride * cap);
        if (!c->d_csum) {
            cap = n_chunks;
            c->d_csum = (double*)c->arena.alloc(sizeof(double) * kSumStride * cap);
        }
        if (!c->d_csum) {
            c->chunks_cap = 0;
            return fail(MBPT_ENOMEM, "arena exhausted (chunk sums)");
        }
        c->chunks_cap = cap;
        changed = true;
    }
    if (hist_floats > c->hist_cap) {
        size_t cap = std::max(hist_floats, c->hist_cap + c->hist_cap / 2);
        c->arena.release(c->d_chist);
        c->d_chist = (float*)c->arena.alloc(sizeof(float) * cap);
        if (!c->d_chist) {
            cap = hist_floats;
            c->d_chist = (float*)c->arena.alloc(sizeof(float) * cap);
        }
        if (!c->d_chist) {
            c->hist_cap = 0;
            return fail(MBPT_ENOMEM, "arena exhausted (chunk histograms)");
        }
        c->hist_cap = cap;
        changed = true;
    }
    if (changed) invalidate_graph(c);
    return MBPT_OK;
}

// The iteration as a graph: reset the chunk counters, one k_iterate launch per non-empty part of the
// batch (bit p of `parts`), k_finalize.  Re-captured when the set of non-empty parts changes.
int capture_graph(mbpt_ctx* c, unsigned parts) {
    if (c->graph && c->graph_parts == parts) return MBPT_OK;
    invalidate_graph(c);
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(c->d_hdr->part_counter, 0, kParts * sizeof(uint32_t), c->stream);
    cudaEventRecordWithFlags(c->ev[0], c->stream, cudaEventRecordExternal);
    const KernelVariant& kv = kVariants[c->variant];
    for (int p = 0; p < kParts; ++p)
        if (parts & (1u << p))
            kv.fn[p]<<<c->variant_blocks[c->variant][p], kv.tpb, kv.smem[p], c->stream>>>(c->d_hdr, c->d_items,
                                                                                          c->d_csum, c->d_chist);
    cudaEventRecordWithFlags(c->ev[1], c->stream, cudaEventRecordExternal);
    k_finalize<<<c->finalize_blocks, 256, 0, c->stream>>>(c->d_hdr, c->d_items, c->d_csum, c->d_chist,
                                                         c->d_last_hist);
    cudaEventRecordWithFlags(c->ev[2], c->stream, cudaEventRecordExternal);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess) return fail(MBPT_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph = nullptr;
        return fail(MBPT_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    c->graph_parts = parts;
    return MBPT_OK;
}

int check_device_error(mbpt_ctx* c) {
    if (!c->d_hdr) return MBPT_OK;
    uint32_t err = 0;
    CUDA_TRY(cudaMemcpyAsync(&err, &c->d_hdr->error, sizeof(err), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (err) return fail(MBPT_EDEVICE, "a kernel reported an out-of-range index (error word " + std::to_string(err) + ")");
    return MBPT_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* mbpt_last_error(void) { return g_err.c_str(); }

int mbpt_ctx_create(mbpt_ctx** out, int device, void* arena, size_t arena_bytes, void* cuda_stream) {
    if (!out || arena_bytes < (1u << 20)) return fail(MBPT_EINVAL, "ctx_create: out is NULL or arena < 1 MiB");
    if (arena && ((uintptr_t)arena & 255)) return fail(MBPT_EINVAL, "ctx_create: arena must be 256-byte aligned");
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(MBPT_EINVAL, "ctx_create: no such device");
    DeviceGuard dg(device);
    mbpt_ctx* c = new (std::nothrow) mbpt_ctx();
    if (!c) return fail(MBPT_ENOMEM, "ctx_create: host allocation");
    c->device = device;
    for (int o = 0; o <= MBPT_MAX_DEVICE_ORDER; ++o) c->spt[o] = kDefaultSpt[o];
    cudaDeviceProp p;
    cudaError_t e = cudaGetDeviceProperties(&p, device);
    if (e != cudaSuccess) {
        delete c;
        return fail(MBPT_ECUDA, std::string("cudaGetDeviceProperties: ") + cudaGetErrorString(e));
    }
    c->sms = p.multiProcessorCount;
    char* base = (char*)arena;
    if (!base) {
        e = cudaMalloc((void**)&base, arena_bytes);
        if (e != cudaSuccess) {
            delete c;
            return fail(MBPT_ENOMEM, std::string("cudaMalloc arena: ") + cudaGetErrorString(e));
        }
        c->own_arena = true;
    }
    c->arena.init(base, arena_bytes);
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            if (c->own_arena) cudaFree(base);
            delete c;
            return fail(MBPT_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    for (int v = 0; v < kNumVariants; ++v) {
        const KernelVariant& kv = kVariants[v];
        for (int p = 0; p < kParts; ++p) {
            int per_sm = 0;
            e = cudaFuncSetAttribute(kv.fn[p], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kv.smem[p]);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kv.fn[p], kv.tpb, kv.smem[p]);
            if (e != cudaSuccess || per_sm < 1) {
                if (c->own_stream) cudaStreamDestroy(c->stream);
                if (c->own_arena) cudaFree(base);
                delete c;
                return fail(MBPT_ECUDA, std::string("k_iterate occupancy: ") + cudaGetErrorString(e));
            }
            c->variant_blocks[v][p] = per_sm * c->sms;
        }
    }
    c->finalize_blocks = 2 * c->sms;
    for (int i = 0; i < 3; ++i) {
        e = cudaEventCreate(&c->ev[i]);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(c->ev[j]);
            if (c->own_stream) cudaStreamDestroy(c->stream);
            if (c->own_arena) cudaFree(base);
            delete c;
            return fail(MBPT_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
        }
    }
    *out = c;
    return MBPT_OK;
}

int mbpt_ctx_destroy(mbpt_ctx* c) {
    if (!c) return fail(MBPT_EINVAL, "ctx_destroy: NULL");
    DeviceGuard dg(c->device);
    cudaStreamSynchronize(c->stream);
    invalidate_graph(c);
    for (mbpt_diag* d : c->diags) delete d;
    c->diags.clear();
    if (c->own_arena) cudaFree(c->arena.base);
    if (c->h_gather) cudaFreeHost(c->h_gather);
    for (int i = 0; i < 3; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return MBPT_OK;
}

int mbpt_ctx_last_timing(mbpt_ctx* c, double* iterate_ms, double* finalize_ms) {
    if (!c || !iterate_ms || !finalize_ms) return fail(MBPT_EINVAL, "last_timing: NULL argument");
    if (!c->graph) return fail(MBPT_EINVAL, "last_timing: no iteration has run");
    DeviceGuard dg(c->device);
    CUDA_TRY(cudaEventSynchronize(c->ev[2]));
    float a = 0.0f, b = 0.0f;
    CUDA_TRY(cudaEventElapsedTime(&a, c->ev[0], c->ev[1]));
    CUDA_TRY(cudaEventElapsedTime(&b, c->ev[1], c->ev[2]));
    *iterate_ms = a;
    *finalize_ms = b;
    return MBPT_OK;
}

int mbpt_ctx_stream(const mbpt_ctx* c, void** stream) {
    if (!c || !stream) return fail(MBPT_EINVAL, "ctx_stream: NULL argument");
    *stream = (void*)c->stream;
    return MBPT_OK;
}

int mbpt_ctx_mem(const mbpt_ctx* c, size_t* used, size_t* largest_free) {
    if (!c || !used || !largest_free) return fail(MBPT_EINVAL, "ctx_mem: NULL argument");
    *used = c->arena.in_use();
    *largest_free = c->arena.largest_free();
    return MBPT_OK;
}

int mbpt_diag_bytes(const mbpt_diagram_desc* desc, const mbpt_vegas_cfg* cfg, size_t* bytes) {
    if (!desc || !cfg || !bytes) return fail(MBPT_EINVAL, "diag_bytes: NULL argument");
    if (desc->n_chords < 1 || desc->n_chords > MBPT_MAX_CHORDS || cfg->n_bins < 2 || cfg->n_bins > MBPT_MAX_BINS)
        return fail(MBPT_EINVAL, "diag_bytes: invalid sizes");
    *bytes = state_block_bytes(3 * desc->n_chords, cfg->n_bins);
    return MBPT_OK;
}

int mbpt_group_bytes(const mbpt_diagram_desc* descs, int k, const mbpt_vegas_cfg* cfg, size_t* bytes) {
    if (!descs || !cfg || !bytes) return fail(MBPT_EINVAL, "group_bytes: NULL argument");
    if (k < 1 || k > MBPT_MAX_GROUP) return fail(MBPT_EINVAL, "group_bytes: member count must be 1..MBPT_MAX_GROUP");
    if (descs[0].n_chords < 1 || descs[0].n_chords > MBPT_MAX_CHORDS || cfg->n_bins < 2 || cfg->n_bins > MBPT_MAX_BINS)
        return fail(MBPT_EINVAL, "group_bytes: invalid sizes");
    *bytes = state_block_bytes(3 * descs[0].n_chords, cfg->n_bins, k);
    return MBPT_OK;
}

int mbpt_kernel_variants(int* tpb, int* minb, int cap, int* count) {
    if (!count) return fail(MBPT_EINVAL, "kernel_variants: NULL count");
    *count = kNumVariants;
    if (!tpb || !minb) return MBPT_OK;
    if (cap < kNumVariants) return fail(MBPT_ENOMEM, "kernel_variants: cap too small");
    for (int v = 0; v < kNumVariants; ++v) {
        tpb[v] = kVariants[v].tpb;
        minb[v] = kVariants[v].minb;
    }
    return MBPT_OK;
}

int mbpt_ctx_set_kernel(mbpt_ctx* c, int tpb, int minb) {
    if (!c) return fail(MBPT_EINVAL, "set_kernel: NULL context");
    for (int v = 0; v < kNumVariants; ++v)
        if (kVariants[v].tpb == tpb && kVariants[v].minb == minb) {
            if (v != c->variant) {
                DeviceGuard dg(c->device);
                cudaStreamSynchronize(c->stream);
                invalidate_graph(c);
                c->variant = v;
            }
            return MBPT_OK;
        }
    return fail(MBPT_EINVAL, "set_kernel: no compiled variant with this shape (see mbpt_kernel_variants)");
}

int mbpt_ctx_set_launch(mbpt_ctx* c, int order, int spt) {
    if (!c || order < 2 || order > MBPT_MAX_DEVICE_ORDER) return fail(MBPT_EINVAL, "set_launch: bad order");
    if (spt < 1 || spt > 256) return fail(MBPT_EINVAL, "set_launch: samples_per_thread must be 1..256");
    c->spt[order] = spt;
    return MBPT_OK;
}

int mbpt_ctx_set_hist_layout(mbpt_ctx* c, int layout) {
    if (!c || (layout != MBPT_HIST_WARP_F32 && layout != MBPT_HIST_BLOCK_F64))
        return fail(MBPT_EINVAL, "set_hist_layout: bad argument");
    c->hist_layout = layout;
    return MBPT_OK;
}

int mbpt_ctx_get_hist_layout(const mbpt_ctx* c, int* layout) {
    if (!c || !layout) return fail(MBPT_EINVAL, "get_hist_layout: NULL argument");
    *layout = c->hist_layout;
    return MBPT_OK;
}

int mbpt_ctx_set_spin_sum(mbpt_ctx* c, int strategy) {
    if (!c || (strategy != MBPT_SPIN_TABLE && strategy != MBPT_SPIN_FOLD))
        return fail(MBPT_EINVAL, "set_spin_sum: bad argument");
    c->spin_sum = strategy;
    return MBPT_OK;
}

int mbpt_ctx_get_spin_sum(const mbpt_ctx* c, int* strategy) {
    if (!c || !strategy) return fail(MBPT_EINVAL, "get_spin_sum: NULL argument");
    *strategy = c->spin_sum;
    return MBPT_OK;
}

int mbpt_ctx_get_launch(const mbpt_ctx* c, int order, int* tpb, int* minb, int* spt) {
    if (!c || !tpb || !minb || !spt || order < 2 || order > MBPT_MAX_DEVICE_ORDER)
        return fail(MBPT_EINVAL, "get_launch: bad argument");
    *tpb = kVariants[c->variant].tpb;
    *minb = kVariants[c->variant].minb;
    *spt = c->spt[order];
    return MBPT_OK;
}

static int create_integral(mbpt_ctx* c, const mbpt_diagram_desc* descs, int k, const double* scale,
                           const mbpt_physics* ph, const mbpt_vegas_cfg* cfg, mbpt_diag** out, const char* who) {
    std::vector<DiagRec> recs((size_t)k);
    char err[256] = {0};
    for (int m = 0; m < k; ++m) {
        // group members are aligned: hole chords first, so that all of them see the same loop momenta
        mbpt_diagram_desc dm = descs[m];
        if (k > 1) hole_chords_first(dm);
        int st = compile_record(dm, *ph, *cfg, &recs[m], err, sizeof(err));
        if (st) return fail(st, std::string(who) + ": member " + std::to_string(m) + ": " + err);
        if (recs[m].order != recs[0].order)
            return fail(MBPT_EINVAL, std::string(who) + ": members must have the same order");
        if (scale) {
            if (!std::isfinite(scale[m])) return fail(MBPT_EINVAL, std::string(who) + ": non-finite member scale");
            set_pref(&recs[m], recs[m].pref * scale[m]);
        }
    }
    DeviceGuard dg(c->device);
    const int d = recs[0].d, nb = recs[0].nb;
    std::vector<double> hf;
    std::vector<float> hff;
    void* d_hf = nullptr;
    if (ph->spectrum == 1) {
        int st = build_hf_table(*ph, hf, err, sizeof(err));
        if (st) return fail(st, std::string(who) + ": " + err);
        hff.resize(hf.size());
        for (size_t i = 0; i < hf.size(); ++i) hff[i] = (float)hf[i];
        const size_t fb = sizeof(double) * hf.size();
        d_hf = c->arena.alloc(fb + sizeof(float) * hff.size());
        if (!d_hf) return fail(MBPT_ENOMEM, std::string(who) + ": arena exhausted (spectrum table)");
        cudaError_t e1 = cudaMemcpyAsync(d_hf, hf.data(), fb, cudaMemcpyHostToDevice, c->stream);
        if (e1 == cudaSuccess)
            e1 = cudaMemcpyAsync((char*)d_hf + fb, hff.data(), sizeof(float) * hff.size(), cudaMemcpyHostToDevice,
                                 c->stream);
        if (e1 != cudaSuccess) {
            c->arena.release(d_hf);
            return fail(MBPT_ECUDA, std::string(who) + " spectrum upload: " + cudaGetErrorString(e1));
        }
        for (int m = 0; m < k; ++m) {
            recs[m].hf_tab = (const double*)d_hf;
            recs[m].hf_tab_f = (const float*)((char*)d_hf + fb);
        }
    }
    char* blk = (char*)c->arena.alloc(state_block_bytes(d, nb, k));
    if (!blk) {
        c->arena.release(d_hf);
        return fail(MBPT_ENOMEM, std::string(who) + ": arena exhausted");
    }
    mbpt_diag* g = new (std::nothrow) mbpt_diag();
    if (!g) {
        c->arena.release(blk);
        return fail(MBPT_ENOMEM, std::string(who) + ": host allocation");
    }
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t rec_bytes = up(sizeof(DiagRec) * (size_t)k);
    g->ctx = c;
    g->desc = descs[0];
    g->phys = *ph;
    g->cfg = *cfg;
    g->d = d;
    g->nb = nb;
    g->n_members = k;
    g->d_hf = d_hf;
    g->d_rec = (DiagRec*)blk;
    g->d_state = (DiagState*)(blk + rec_bytes);
    g->d_grid = (double*)(blk + rec_bytes + up(sizeof(DiagState)));
    g->d_last_hist = (double*)((char*)g->d_grid + up(sizeof(double) * d * (nb + 1)));
    std::vector<double> grid((size_t)d * (nb + 1));
    for (int a = 0; a < d; ++a)
        for (int i = 0; i <= nb; ++i) grid[(size_t)a * (nb + 1) + i] = (double)i / nb;
    DiagState s0;
    memset(&s0, 0, sizeof(s0));
    cudaError_t e = cudaMemcpyAsync(g->d_rec, recs.data(), sizeof(DiagRec) * (size_t)k, cudaMemcpyHostToDevice,
                                    c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->d_state, &s0, sizeof(s0), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->d_grid, grid.data(), sizeof(double) * grid.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_last_hist, 0, sizeof(double) * d * nb, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->arena.release(blk);
        c->arena.release(d_hf);
        delete g;
        return fail(MBPT_ECUDA, std::string(who) + " upload: " + cudaGetErrorString(e));
    }
    c->diags.insert(g);
    *out = g;
    return MBPT_OK;
}

int mbpt_create_diagram(mbpt_ctx* c, const mbpt_diagram_desc* desc, const mbpt_physics* ph,
                        const mbpt_vegas_cfg* cfg, mbpt_diag** out) {
    if (!c || !desc || !ph || !cfg || !out) return fail(MBPT_EINVAL, "create_diagram: NULL argument");
    return create_integral(c, desc, 1, nullptr, ph, cfg, out, "create_diagram");
}

int mbpt_create_group(mbpt_ctx* c, const mbpt_diagram_desc* descs, int k, const double* scale,
                      const mbpt_physics* ph, const mbpt_vegas_cfg* cfg, mbpt_diag** out) {
    if (!c || !descs || !ph || !cfg || !out) return fail(MBPT_EINVAL, "create_group: NULL argument");
    if (k < 1 || k > MBPT_MAX_GROUP) return fail(MBPT_EINVAL, "create_group: member count must be 1..MBPT_MAX_GROUP");
    return create_integral(c, descs, k, scale, ph, cfg, out, "create_group");
}

int mbpt_set_config(mbpt_diag* g, const mbpt_vegas_cfg* cfg) {
    if (!g || !cfg || !g->ctx || !g->ctx->diags.count(g)) return fail(MBPT_EINVAL, "set_config: bad argument");
    const mbpt_vegas_cfg& o = g->cfg;
    if (cfg->n_bins != o.n_bins || cfg->precision != o.precision || cfg->seed != o.seed ||
        cfg->stream_id != o.stream_id || cfg->alpha != o.alpha || cfg->n_shifts != o.n_shifts ||
        cfg->combine != o.combine || cfg->near_band != o.near_band ||
        (o.n_shifts && (cfg->shift[0] != o.shift[0] || cfg->shift[1] != o.shift[1] || cfg->shift[2] != o.shift[2])))
        return fail(MBPT_EINVAL, "set_config: only samples_per_iter, freeze_after, train_iters and the targets may change");
    if (cfg->samples_per_iter < 2 || cfg->samples_per_iter >= (1ull << 32) || !(cfg->target_rel >= 0.0) ||
        !(cfg->target_abs >= 0.0))
        return fail(MBPT_EINVAL, "set_config: invalid samples or targets");
    g->cfg.samples_per_iter = cfg->samples_per_iter;
    g->cfg.freeze_after = cfg->freeze_after;
    g->cfg.target_rel = cfg->target_rel;
    g->cfg.target_abs = cfg->target_abs;
    g->cfg.train_iters = cfg->train_iters;
    return MBPT_OK;
}

int mbpt_destroy_diagram(mbpt_diag* g) {
    if (!g || !g->ctx) return fail(MBPT_EINVAL, "destroy_diagram: NULL");
    mbpt_ctx* c = g->ctx;
    if (!c->diags.count(g)) return fail(MBPT_EINVAL, "destroy_diagram: unknown integral");
    DeviceGuard dg(c->device);
    cudaStreamSynchronize(c->stream);   // no queued work may still reference it
    c->arena.release(g->d_rec);
    c->arena.release(g->d_hf);
    c->diags.erase(g);
    delete g;
    return MBPT_OK;
}

int mbpt_vegas_iterate(mbpt_ctx* c, mbpt_diag* const* diags, int k, int n_iters) {
    if (!c || k < 0 || n_iters < 0 || (k > 0 && !diags)) return fail(MBPT_EINVAL, "vegas_iterate: bad argument");
    if (k == 0 || n_iters == 0) return MBPT_OK;
    DeviceGuard dg(c->device);
    c->h_items.clear();
    c->h_last_hist.clear();
    uint64_t chunk = 0;
    int stride = 0;
    std::set<mbpt_diag*> seen;
    for (int i = 0; i < k; ++i) {
        mbpt_diag* g = diags[i];
        if (!g || !c->diags.count(g)) return fail(MBPT_EINVAL, "vegas_iterate: integral not owned by this context");
        if (!seen.insert(g).second) return fail(MBPT_EINVAL, "vegas_iterate: integral listed twice");
        stride = std::max(stride, g->d * g->nb);
    }
    // the batch's parts in kernel order (bit 0: regulator, bit 1: group, bit 2: sixth order), each in call order
    auto part_of = [](const mbpt_diag* g) {
        return (g->cfg.n_shifts != 0 ? kPartReg : 0) | (g->n_members > 1 ? kPartGrp : 0) |
               (g->desc.order == 6 ? kPartO6 : 0);
    };
    std::vector<mbpt_diag*> order_v;
    order_v.reserve((size_t)k);
    for (int part = 0; part < kParts; ++part)
        for (int i = 0; i < k; ++i)
            if (part_of(diags[i]) == part) order_v.push_back(diags[i]);
    uint32_t part_items[kParts] = {}, part_chunks[kParts] = {};
    for (int i = 0; i < k; ++i) {
        mbpt_diag* g = order_v[(size_t)i];
        const int part = part_of(g);
        WorkItem w;
        memset(&w, 0, sizeof(w));
        w.rec = g->d_rec;
        w.state = g->d_state;
        w.grid = g->d_grid;
        w.samples = g->cfg.samples_per_iter;
        w.seed = g->cfg.seed;
        w.stream_id = g->cfg.stream_id;
        w.n_members = (uint32_t)g->n_members;
        // a group keeps per-sample member sums in shared-memory slots: 16 samples per thread, 3 with the
        // regulator (five slots per sample)
        w.spt = g->n_members > 1 ? (g->cfg.n_shifts ? kGroupSlotsReg / (1 + kComp) : kGroupSlotsPlain)
                                 : c->spt[g->desc.order];
        const uint64_t cs = (uint64_t)kVariants[c->variant].tpb * (uint64_t)w.spt;
        w.n_chunks = (uint32_t)((w.samples + cs - 1) / cs);
        w.chunk_begin = (uint32_t)chunk;
        w.freeze_after = g->cfg.freeze_after;
        w.alpha = g->cfg.alpha;
        w.target_rel = g->cfg.target_rel;
        w.target_abs = g->cfg.target_abs;
        w.train_iters = g->cfg.train_iters;
        w.combine = g->cfg.combine;
        w.hist_layout = (uint32_t)c->hist_layout;
        w.spin_sum = (uint32_t)c->spin_sum;
        w.hist_stride = stride;
        chunk += w.n_chunks;
        if (chunk >= (1ull << 31)) return fail(MBPT_EINVAL, "vegas_iterate: batch too large");
        part_items[part] += 1;
        part_chunks[part] += w.n_chunks;
        c->h_items.push_back(w);
        c->h_last_hist.push_back(g->d_last_hist);
    }
    int st = ensure_batch_buffers(c, (size_t)k, (size_t)chunk, (size_t)chunk * (size_t)stride);
    if (st) return st;
    WorkHeader h;
    memset(&h, 0, sizeof(h));
    h.n_items = (uint32_t)k;
    h.total_chunks = (uint32_t)chunk;
    h.hist_floats = (uint64_t)chunk * (uint64_t)stride;
    for (int p = 0; p < kParts; ++p) {
        h.part_items[p] = part_items[p];
        h.part_chunks[p] = part_chunks[p];
    }
    CUDA_TRY(cudaMemcpyAsync(c->d_items, c->h_items.data(), sizeof(WorkItem) * k, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->d_last_hist, c->h_last_hist.data(), sizeof(double*) * k, cudaMemcpyHostToDevice,
                             c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->d_hdr, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    unsigned parts = 0;
    for (int p = 0; p < kParts; ++p)
        if (part_items[p]) parts |= 1u << p;
    st = capture_graph(c, parts);
    if (st) return st;
    for (int it = 0; it < n_iters; ++it) CUDA_TRY(cudaGraphLaunch(c->graph, c->stream));
    CUDA_TRY(cudaGetLastError());
    return MBPT_OK;
}

int mbpt_estimate(const mbpt_diag* g, mbpt_result* out) {
    if (!g || !out || !g->ctx) return fail(MBPT_EINVAL, "estimate: NULL argument");
    mbpt_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    int st = check_device_error(c);
    if (st) return st;
    DiagState s;
    CUDA_TRY(cudaMemcpyAsync(&s, g->d_state, offsetof(DiagState, hist_mean), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    out->mean = s.mean;
    out->sigma = s.sigma;
    out->chi2_dof = s.chi2;
    out->last_mean = s.last_mean;
    out->last_sigma = s.last_var > 0.0 ? sqrt(s.last_var) : 0.0;
    out->n_iter = s.iter;
    out->n_evals = s.n_evals;
    out->converged = s.converged;
    out->status = s.status;
    return MBPT_OK;
}

int mbpt_estimate_batch(mbpt_diag* const* diags, int k, mbpt_result* out) {
    if (k < 0 || (k > 0 && (!diags || !out))) return fail(MBPT_EINVAL, "estimate_batch: bad argument");
    if (k == 0) return MBPT_OK;
    mbpt_ctx* c = diags[0] ? diags[0]->ctx : nullptr;
    if (!c) return fail(MBPT_EINVAL, "estimate_batch: NULL integral");
    for (int i = 0; i < k; ++i)
        if (!diags[i] || diags[i]->ctx != c || !c->diags.count(diags[i]))
            return fail(MBPT_EINVAL, "estimate_batch: integrals must belong to one context");
    DeviceGuard dg(c->device);
    int st = check_device_error(c);
    if (st) return st;
    // the states' heads (estimate, error, counters) gathered on the device by one kernel and read back with
    // one copy; per-integral copies (about 10 us each) only if the gather buffers cannot be had
    constexpr size_t kHead = offsetof(DiagState, hist_mean);
    static_assert(kHead % 16 == 0, "the state head is copied as 16-byte words");
    if ((size_t)k > c->gather_cap) {
        const size_t cap = std::max((size_t)k, 2 * c->gather_cap);
        c->arena.release(c->d_gather_src);
        c->arena.release(c->d_gather_out);
        if (c->h_gather) cudaFreeHost(c->h_gather);
        c->h_gather = nullptr;
        c->gather_cap = 0;
        c->d_gather_src = (const DiagState**)c->arena.alloc(sizeof(DiagState*) * cap);
        c->d_gather_out = (uint4*)c->arena.alloc(kHead * cap);
        if (c->d_gather_src && c->d_gather_out &&
            cudaMallocHost(&c->h_gather, (sizeof(DiagState*) + kHead) * cap) == cudaSuccess)
            c->gather_cap = cap;
        else
            cudaGetLastError();
    }
    std::vector<DiagState> hs;
    const unsigned char* heads = nullptr;
    if ((size_t)k <= c->gather_cap) {
        const DiagState** hp = (const DiagState**)c->h_gather;
        unsigned char* hh = (unsigned char*)c->h_gather + sizeof(DiagState*) * c->gather_cap;
        for (int i = 0; i < k; ++i) hp[i] = diags[i]->d_state;
        CUDA_TRY(cudaMemcpyAsync(c->d_gather_src, hp, sizeof(DiagState*) * k, cudaMemcpyHostToDevice, c->stream));
        const int words = (int)(kHead / 16);
        k_gather_heads<<<(k * words + 255) / 256, 256, 0, c->stream>>>(c->d_gather_src, k, words, c->d_gather_out);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(hh, c->d_gather_out, kHead * k, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        heads = hh;
    } else {
        hs.resize((size_t)k);
        for (int i = 0; i < k; ++i)
            CUDA_TRY(cudaMemcpyAsync(&hs[i], diags[i]->d_state, kHead, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    for (int i = 0; i < k; ++i) {
        DiagState sh;
        if (heads) memcpy(&sh, heads + kHead * i, kHead);
        const DiagState& s = heads ? sh : hs[i];
        out[i].mean = s.mean;
        out[i].sigma = s.sigma;
        out[i].chi2_dof = s.chi2;
        out[i].last_mean = s.last_mean;
        out[i].last_sigma = s.last_var > 0.0 ? sqrt(s.last_var) : 0.0;
        out[i].n_iter = s.iter;
        out[i].n_evals = s.n_evals;
        out[i].converged = s.converged;
        out[i].status = s.status;
    }
    return MBPT_OK;
}

int mbpt_estimate_shifts(const mbpt_diag* g, double mean[4], double sigma[4]) {
    if (!g || !mean || !sigma || !g->ctx) return fail(MBPT_EINVAL, "estimate_shifts: NULL argument");
    if (!g->cfg.n_shifts) return fail(MBPT_EINVAL, "estimate_shifts: the integral has no regulator shifts");
    mbpt_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    int st = check_device_error(c);
    if (st) return st;
    double buf[4 * kComp];
    CUDA_TRY(cudaMemcpyAsync(buf, g->d_state->comp_inv_var, sizeof(buf), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int q = 0; q < kComp; ++q) {
        mean[q] = buf[2 * kComp + q];
        sigma[q] = buf[3 * kComp + q];
    }
    return MBPT_OK;
}

// checkpoint image: header, DiagState, grid, last histogram
struct StateHeader {
    uint32_t magic, version;
    int32_t d, nb, order;
    int32_t pad;
};
static const uint32_t kMagic = 0x4D425054u;   // "MBPT"
static const uint32_t kStateVersion = 2u;      // 2: DiagState with the pooled evaluation-phase sums

int mbpt_get_state(const mbpt_diag* g, void* buf, size_t cap, size_t* need) {
    if (!g || !need) return fail(MBPT_EINVAL, "get_state: NULL argument");
    const size_t n_grid = (size_t)g->d * (g->nb + 1), n_hist = (size_t)g->d * g->nb;
    const size_t bytes = sizeof(StateHeader) + sizeof(DiagState) + sizeof(double) * (n_grid + n_hist);
    *need = bytes;
    if (!buf) return MBPT_OK;
    if (cap < bytes) return fail(MBPT_ENOMEM, "get_state: buffer too small");
    mbpt_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    char* p = (char*)buf;
    StateHeader h = {kMagic, kStateVersion, g->d, g->nb, g->desc.order, 0};
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    CUDA_TRY(cudaMemcpyAsync(p, g->d_state, sizeof(DiagState), cudaMemcpyDeviceToHost, c->stream));
    p += sizeof(DiagState);
    CUDA_TRY(cudaMemcpyAsync(p, g->d_grid, sizeof(double) * n_grid, cudaMemcpyDeviceToHost, c->stream));
    p += sizeof(double) * n_grid;
    CUDA_TRY(cudaMemcpyAsync(p, g->d_last_hist, sizeof(double) * n_hist, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return MBPT_OK;
}

int mbpt_set_state(mbpt_diag* g, const void* buf, size_t len) {
    if (!g || !buf) return fail(MBPT_EINVAL, "set_state: NULL argument");
    const size_t n_grid = (size_t)g->d * (g->nb + 1), n_hist = (size_t)g->d * g->nb;
    const size_t bytes = sizeof(StateHeader) + sizeof(DiagState) + sizeof(double) * (n_grid + n_hist);
    if (len != bytes) return fail(MBPT_EINVAL, "set_state: wrong image size");
    StateHeader h;
    memcpy(&h, buf, sizeof(h));
    if (h.magic != kMagic || h.version != kStateVersion || h.d != g->d || h.nb != g->nb || h.order != g->desc.order)
        return fail(MBPT_EINVAL, "set_state: image does not match this integral");
    const char* p = (const char*)buf + sizeof(h);
    DiagState s;
    memcpy(&s, p, sizeof(s));
    // validate the grid: monotone from 0 to 1
    const double* grid = (const double*)(p + sizeof(DiagState));
    for (int a = 0; a < g->d; ++a) {
        const double* e = grid + (size_t)a * (g->nb + 1);
        if (e[0] != 0.0 || e[g->nb] != 1.0) return fail(MBPT_EINVAL, "set_state: grid must span [0, 1]");
        for (int i = 0; i < g->nb; ++i)
            if (!(e[i + 1] >= e[i])) return fail(MBPT_EINVAL, "set_state: grid must be non-decreasing");
    }
    mbpt_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    CUDA_TRY(cudaMemcpyAsync(g->d_state, p, sizeof(DiagState), cudaMemcpyHostToDevice, c->stream));
    p += sizeof(DiagState);
    CUDA_TRY(cudaMemcpyAsync(g->d_grid, p, sizeof(double) * n_grid, cudaMemcpyHostToDevice, c->stream));
    p += sizeof(double) * n_grid;
    CUDA_TRY(cudaMemcpyAsync(g->d_last_hist, p, sizeof(double) * n_hist, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return MBPT_OK;
}

int mbpt_dump_samples(mbpt_diag* g, int64_t iter, int64_t first, int64_t count, double* x, double* w) {
    if (!g || !w || iter < 0 || iter >= (1ll << 32) || first < 0 || count < 0 || first + count > (1ll << 32))
        return fail(MBPT_EINVAL, "dump_samples: bad argument");
    if (count == 0) return MBPT_OK;
    mbpt_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    double* dx = x ? (double*)c->arena.alloc(sizeof(double) * (size_t)count * g->d) : nullptr;
    double* dw = (double*)c->arena.alloc(sizeof(double) * (size_t)count);
    if ((x && !dx) || !dw) {
        c->arena.release(dx);
        c->arena.release(dw);
        return fail(MBPT_ENOMEM, "dump_samples: arena exhausted");
    }
    const int blocks = (int)((count + 255) / 256);
    k_dump<<<blocks, 256, 0, c->stream>>>(g->d_rec, g->n_members, g->d_grid, g->cfg.seed, g->cfg.stream_id,
                                          (uint32_t)iter, (uint64_t)first, (uint64_t)count, (uint32_t)c->spin_sum, dx,
                                          dw);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && x)
        e = cudaMemcpyAsync(x, dx, sizeof(double) * (size_t)count * g->d, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w, dw, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->arena.release(dx);
    c->arena.release(dw);
    if (e != cudaSuccess) return fail(MBPT_ECUDA, std::string("dump_samples: ") + cudaGetErrorString(e));
    return MBPT_OK;
}

int mbpt_philox_device(mbpt_ctx* c, const uint32_t ctr[4], const uint32_t key[2], int64_t count, uint32_t* out) {
    if (!c || !ctr || !key || !out || count < 0 || count > (1ll << 26)) return fail(MBPT_EINVAL, "philox_device: bad argument");
    if (count == 0) return MBPT_OK;
    DeviceGuard dg(c->device);
    uint32_t* d = (uint32_t*)c->arena.alloc(sizeof(uint32_t) * 4 * (size_t)count);
    if (!d) return fail(MBPT_ENOMEM, "philox_device: arena exhausted");
    k_philox<<<(unsigned)((count + 255) / 256), 256, 0, c->stream>>>(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1],
                                                                   (uint64_t)count, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, d, sizeof(uint32_t) * 4 * (size_t)count, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->arena.release(d);
    if (e != cudaSuccess) return fail(MBPT_ECUDA, std::string("philox_device: ") + cudaGetErrorString(e));
    return MBPT_OK;
}

}  // extern "C"

static_assert(sizeof(WorkItem) == 112 && sizeof(WorkHeader) == 128,
              "work table layout changed: update the binding's transfer sizes (mbpt.py WORK_ITEM_BYTES, WORK_HEADER_BYTES)");

// ---------------------------------------------------------------------------
// Allocation-free single iteration (mbpt_vegas_iteration_noalloc).
//
// Some callers must not allocate device memory once they are running: a process whose device
// memory is owned by another allocator (a framework's caching allocator, a fixed per-tenant
// budget), or a latency-critical loop in which cudaMalloc/cudaFree, with their implicit device
// synchronisation, are not acceptable.  For them the chunk slots, work table, compiled record and
// per-integral state that mbpt_vegas_iterate keeps in its arena live in one fixed-size device
// array defined here; the caller passes only the grid (input) and the result buffer (output).
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = 32ull << 20;   // per device, held from load to process exit
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
constexpr int kNoAllocMaxDevices = 64;

struct NoAllocDevice {
    bool ready = false;
    unsigned char* ptr = nullptr;   // device address of g_noalloc_scratch on this device
    int blocks[2] = {0, 0};         // persistent grids of k_iterate: orders 2..5, sixth order
};
// the k_iterate kernels of a fresh context's default launch shape (256 threads, 2 blocks per SM) for plain
// integrals of orders 2..5 and of the sixth order
const IterateFn kNoAllocFn[2] = {MBPT_K_ITERATE(256, 2, 0), MBPT_K_ITERATE(256, 2, 4)};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];

// Once per device, with that device current: the device address of the scratch array (its name
// in host code is only a host-side stand-in) and the launch attributes of k_iterate.
int noalloc_setup(int device, NoAllocDevice** out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDevice& d = g_noalloc_dev[device];
    if (!d.ready) {
        void* p = nullptr;
        CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        int sms = 0;
        CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        for (int k = 0; k < 2; ++k) {
            CUDA_TRY(cudaFuncSetAttribute(kNoAllocFn[k], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sizeof(ChunkSmem)));
            int per_sm = 0;
            CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kNoAllocFn[k], kThreads,
                                                                   sizeof(ChunkSmem)));
            if (per_sm < 1) return fail(MBPT_ECUDA, "noalloc: k_iterate cannot be resident");
            d.blocks[k] = per_sm * sms;
        }
        d.ptr = (unsigned char*)p;
        d.ready = true;
    }
    *out = &d;
    return MBPT_OK;
}

// Fixed-order sums of one integral's chunk slots: out = [sum w, sum w^2, histogram d x nb].  If k_iterate
// set its error word (an out-of-range chunk, a misplaced item or a record no compiled case matches), every
// output is NaN instead.
__global__ void __launch_bounds__(256) k_reduce_noalloc(const WorkHeader* __restrict__ hdr,
                                                       const WorkItem* __restrict__ item,
                                                       const double* __restrict__ csum,
                                                       const float* __restrict__ chist, double* __restrict__ out) {
    __shared__ double red[2][8];
    const WorkItem& W = *item;
    const int tid = threadIdx.x;
    const int nh = W.rec->d * W.rec->nb;
    if (hdr->error != 0u) {
        for (int i = tid; i < 2 + nh; i += blockDim.x) out[i] = __longlong_as_double(0x7FF8000000000000ll);
        return;
    }
    double a = 0.0, b = 0.0;
    for (uint32_t c = tid; c < W.n_chunks; c += blockDim.x) {
        a += csum[kSumStride * (size_t)c];
        b += csum[kSumStride * (size_t)c + 1];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = a;
        red[1][tid >> 5] = b;
    }
    __syncthreads();
    if (tid == 0) {
        double A = 0.0, B = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            A += red[0][w];
            B += red[1][w];
        }
        out[0] = A;
        out[1] = B;
    }
    for (int i = tid; i < nh; i += blockDim.x)
        out[2 + i] = hist_column_sum(chist + i, (size_t)W.hist_stride, W.n_chunks);   // as k_finalize
}

}  // namespace

extern "C" int mbpt_vegas_iteration_noalloc(int device, const mbpt_diagram_desc* desc, const mbpt_physics* ph,
                                            const mbpt_vegas_cfg* cfg, uint32_t iter, const double* grid,
                                            double* out, void* cuda_stream) {
    if (!desc || !ph || !cfg || !grid || !out) return fail(MBPT_EINVAL, "iteration_noalloc: NULL argument");
    if (cfg->n_shifts) return fail(MBPT_EINVAL, "iteration_noalloc: denominator regulator not supported here");
    if (ph->spectrum) return fail(MBPT_EINVAL, "iteration_noalloc: the Hartree-Fock spectrum is not supported here");
    if (device < 0 || device >= kNoAllocMaxDevices) return fail(MBPT_EINVAL, "iteration_noalloc: bad device");
    DiagRec rec;
    char err[256] = {0};
    int st = compile_record(*desc, *ph, *cfg, &rec, err, sizeof(err));
    if (st) return fail(st, std::string("iteration_noalloc: ") + err);
    const int spt = kDefaultSpt[rec.order];   // as a fresh context (256 threads)
    const uint64_t cs = (uint64_t)kThreads * (uint64_t)spt;
    const uint64_t n_chunks = (cfg->samples_per_iter + cs - 1) / cs;
    const size_t nh = (size_t)rec.d * (size_t)rec.nb;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t off_hdr = 0, off_item = up(sizeof(WorkHeader)), off_rec = off_item + up(sizeof(WorkItem));
    const size_t off_state = off_rec + up(sizeof(DiagRec)), off_csum = off_state + up(sizeof(DiagState));
    const size_t off_chist = off_csum + up(sizeof(double) * kSumStride * n_chunks);
    const size_t need = off_chist + sizeof(float) * nh * n_chunks;
    if (need > kNoAllocScratchBytes) {
        const uint64_t per_chunk = 8 * kSumStride + 4 * nh;
        const uint64_t max_chunks = (kNoAllocScratchBytes - off_csum - 512) / per_chunk;
        return fail(MBPT_EINVAL, "iteration_noalloc: " + std::to_string(cfg->samples_per_iter) +
                                     " samples need " + std::to_string(need) + " bytes of scratch, more than the " +
                                     std::to_string(kNoAllocScratchBytes) + "-byte array; at most " +
                                     std::to_string(max_chunks * cs) + " samples per call for this diagram");
    }
    DeviceGuard dg(device);
    NoAllocDevice* nd = nullptr;
    st = noalloc_setup(device, &nd);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char* base = nd->ptr;
    WorkHeader h;
    memset(&h, 0, sizeof(h));          // chunk counter and error word start at zero on every call
    h.n_items = 1;
    h.total_chunks = (uint32_t)n_chunks;
    h.hist_floats = (uint64_t)nh * n_chunks;
    const int part = rec.order == 6 ? kPartO6 : 0;
    h.part_items[part] = 1;
    h.part_chunks[part] = (uint32_t)n_chunks;
    DiagState s0;
    memset(&s0, 0, sizeof(s0));
    s0.iter = (int32_t)iter;
    WorkItem w;
    memset(&w, 0, sizeof(w));
    w.rec = (const DiagRec*)(base + off_rec);
    w.state = (DiagState*)(base + off_state);
    w.grid = const_cast<double*>(grid);
    w.samples = cfg->samples_per_iter;
    w.seed = cfg->seed;
    w.stream_id = cfg->stream_id;
    w.chunk_begin = 0;
    w.n_chunks = (uint32_t)n_chunks;
    w.alpha = cfg->alpha;
    w.spt = spt;
    w.n_members = 1;
    w.hist_stride = (int32_t)nh;
    CUDA_TRY(cudaMemcpyAsync(base + off_hdr, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(base + off_item, &w, sizeof(w), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(base + off_rec, &rec, sizeof(rec), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(base + off_state, &s0, sizeof(s0), cudaMemcpyHostToDevice, s));
    const int kk = part == kPartO6 ? 1 : 0;
    kNoAllocFn[kk]<<<nd->blocks[kk], kThreads, sizeof(ChunkSmem), s>>>((WorkHeader*)(base + off_hdr),
                                                                       (const WorkItem*)(base + off_item),
                                                                       (double*)(base + off_csum),
                                                                       (float*)(base + off_chist));
    CUDA_TRY(cudaGetLastError());
    k_reduce_noalloc<<<1, 256, 0, s>>>((const WorkHeader*)(base + off_hdr), (const WorkItem*)(base + off_item),
                                       (const double*)(base + off_csum), (const float*)(base + off_chist), out);
    CUDA_TRY(cudaGetLastError());
    return MBPT_OK;
}

namespace mbpt {
__global__ void k_dfma_rate(int iters);   // mbpt_k_misc.cu
}

extern "C" int mbpt_fp64_rate(int device, void* cuda_stream, double* ops_per_s) {
    if (!ops_per_s) return fail(MBPT_EINVAL, "fp64_rate: NULL argument");
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(MBPT_EINVAL, "fp64_rate: no such device");
    DeviceGuard dg(device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int blocks = 8 * sms, threads = 256, iters = 4096;   // 2048 resident threads per SM
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    float best = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            k_dfma_rate<<<blocks, threads, 0, s>>>(iters);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(MBPT_ECUDA, std::string("fp64_rate: ") + cudaGetErrorString(e));
    *ops_per_s = 8.0 * (double)iters * (double)threads * (double)blocks / (1e-3 * (double)best);
    return MBPT_OK;
}
