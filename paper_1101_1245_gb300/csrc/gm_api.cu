// C ABI of the gpumcd library (include/gpumcd.h): contexts, device memory
// under an HBM budget, phantoms, plans and the launch sequence of the
// persistent transport kernel.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <numeric>
#include <vector>

#include "gm_common.cuh"
#include "gm_host.h"

using namespace gm;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Phantom {
    int32_t dims[3];
    double voxel[3];
    uint64_t nvox;
    DevBuf vox;     // packed voxel words
    DevBuf rhomax;  // [NMAT] float bits
    DevBuf maj;     // [2G] majorants
};

struct Plan {
    int32_t phantom;
    int32_t particle, beam;
    double energy, cx, cy, field;
    int32_t n_spec;
    uint32_t n_phsp = 0;     // phase-space records (held in `spec`)
    bool e_group = false;    // a spectrum or phase space grouped by energy: claimed highest energies first
    uint64_t seed;
    uint32_t W;
    uint64_t hist_sub = 0;   // histories handed to launch sequences (numbering of the next run)
    uint64_t hist_done = 0;  // histories of completed sequences (what a fold sees)
    int inflight = 0;        // unfinished sequences that include this plan
    bool failed = false;     // a sequence failed: the tally is incomplete until plan_reset
    cudaEvent_t reset_done = nullptr;  // after the last plan_reset's memsets (any stream)
    DevBuf tally;   // [W][nvox] u64
    DevBuf ledger;  // [4] u64
    DevBuf spec;    // [2(n_spec+1)] floats
    gpumcd_run_stats acc;  // counters accumulated over the plan's runs
};

// Device control block of a launch sequence.
struct Control {
    unsigned long long prim_cursor[2];
    unsigned long long qcur[2][NT];  // [buffer][type]
    unsigned long long counters[CNT_N];
    int32_t error;
    int32_t pad;
};

// Scratch and state of one launch sequence (the persistent kernel, then
// relaunches over the overflow queues until they are empty).  Slot 0 serves
// gpumcd_run on the caller's stream; slots 1..GPUMCD_MAX_INFLIGHT serve
// gpumcd_submit on their own streams, so sequences can overlap on the device.
struct Slot {
    DevBuf stacks, hard, queue[2][NT], control, plandev;
    DevBuf order, gcount;  // claim orders of grouped sources, and their sort's bin counts
    Control *h_control = nullptr;  // pinned: the control block after each launch
    PlanDev *h_plandev = nullptr;  // pinned: the sequence's plan table
    cudaStream_t own = nullptr;    // the slot's stream (asynchronous slots)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, done = nullptr;
    bool busy = false;
    int32_t ticket = 0;
    cudaStream_t s = nullptr;  // the stream the sequence runs on
    TransportArgs A;
    int grid = 0, block = 0, bps = 0;
    uint32_t k = 0;  // launches enqueued
    unsigned long long in_count[NT] = {0, 0};
    std::vector<int32_t> ids;
    std::vector<uint64_t> n_hist;
    // GPUMCD_LAUNCH_GRAPH: the first launch of a sequence (plan-table copy,
    // control reset, kernel, control read-back) captured once per launch
    // shape and replayed with the kernel's arguments updated
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphNode_t knode = nullptr;
    int g_grid = 0, g_block = 0, g_bps = 0;
    const void *g_fn = nullptr;  // the transport kernel the graph holds
};

}  // namespace

struct gpumcd_ctx {
    int device = 0;
    int n_sm = 0;
    cudaStream_t stream = nullptr;
    uint64_t budget = 0, used = 0;
    uint64_t cache_max = 32ull << 30;  // without a budget: half the device's memory, at least 32 GB
    bool tables = false;
    int n_mat = 0;
    gpumcd_physics phys{};
    TableGeom geom{};
    Phys dphys{};
    DevBuf tab;
    std::map<int32_t, Phantom> phantoms;
    std::map<int32_t, Plan> plans;
    int32_t next_id = 1;
    gpumcd_launch launch{};
    Slot slot[1 + GPUMCD_MAX_INFLIGHT];
    Control last{};          // control block of the last finished sequence
    bool have_last = false;
    cudaEvent_t order = nullptr;  // orders a submitted sequence after the context stream
    int32_t next_ticket = 1;
    DevBuf fold_tmp;
    std::multimap<size_t, void *> cache;  // freed device blocks by size
    uint64_t cached = 0;
    bool configured = false;
};

namespace {

gpumcd_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GPUMCD_OK;
    if (e == cudaErrorMemoryAllocation) return GPUMCD_ERR_OOM;
    return GPUMCD_ERR_CUDA;
}

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_status(e_);    \
    } while (0)

#define ST(call)                                  \
    do {                                          \
        gpumcd_status s_ = (call);                \
        if (s_ != GPUMCD_OK) return s_;           \
    } while (0)

// Device memory is cached: a freed block goes to a size-keyed free list and
// is handed out again for a request of up to its size (and within a quarter
// of it, plus 1 MB), so steady-state create/open/close/destroy cycles call neither
// cudaMalloc nor cudaFree (which synchronizes the whole device, stalling any
// sequence in flight).  A block enters the cache only when no GPU work on it
// is pending: every caller of dev_free has synchronized the streams that used
// it.  The budget counts live bytes; live + cached bytes stay within it, and
// without a budget the cache keeps at most cache_max bytes: half of the
// device's memory (at least 32 GB), so a working set of tens of GB (the
// tallies of 64 plans) cycles through the cache and never through cudaFree.

void cache_trim(gpumcd_ctx *c, uint64_t limit) {
    while (c->cached > limit && !c->cache.empty()) {
        auto it = std::prev(c->cache.end());  // largest block first
        cudaFree(it->second);
        c->cached -= it->first;
        c->cache.erase(it);
    }
}

void dev_free(gpumcd_ctx *c, DevBuf &b) {
    if (b.p) {
        c->used -= b.bytes;
        c->cache.emplace(b.bytes, b.p);
        c->cached += b.bytes;
        if (c->budget) cache_trim(c, c->budget > c->used ? c->budget - c->used : 0);
        else cache_trim(c, c->cache_max);
    }
    b.p = nullptr;
    b.bytes = 0;
}

gpumcd_status dev_alloc(gpumcd_ctx *c, DevBuf &b, size_t bytes) {
    if (b.p && b.bytes >= bytes) return GPUMCD_OK;
    if (c->budget && c->used - b.bytes + bytes > c->budget) return GPUMCD_ERR_BUDGET;
    dev_free(c, b);
    if (bytes == 0) return GPUMCD_OK;
    auto it = c->cache.lower_bound(bytes);
    if (it != c->cache.end() && it->first <= bytes + bytes / 4 + (1u << 20) &&
        (!c->budget || c->used + it->first <= c->budget)) {
        b.p = it->second;
        b.bytes = it->first;
        c->cached -= it->first;
        c->cache.erase(it);
        c->used += b.bytes;
        return GPUMCD_OK;
    }
    if (c->budget) cache_trim(c, c->budget - c->used - bytes);
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaErrorMemoryAllocation && c->cached) {
        cudaGetLastError();
        cache_trim(c, 0);
        e = cudaMalloc(&b.p, bytes);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return GPUMCD_ERR_OOM;
    }
    b.bytes = bytes;
    c->used += bytes;
    return GPUMCD_OK;
}

cudaStream_t pick(gpumcd_ctx *c, void *stream) { return stream ? (cudaStream_t)stream : c->stream; }

gpumcd_status set_device(gpumcd_ctx *c) {
    CK(cudaSetDevice(c->device));
    return GPUMCD_OK;
}

bool valid_source(const gpumcd_ctx *c, const gpumcd_source *s) {
    if (!s) return false;
    if (s->particle != GPUMCD_PHOTON && s->particle != GPUMCD_ELECTRON) return false;
    if (s->energy_grouping != GPUMCD_ENERGY_UNGROUPED && s->energy_grouping != GPUMCD_ENERGY_GROUPED) return false;
    if (s->beam == GPUMCD_BEAM_PHASE_SPACE)  // records are checked when copied
        return s->n_phase_space >= 1 && s->n_phase_space <= (1 << 24) && s->phase_space;
    if (s->beam != GPUMCD_BEAM_PENCIL && s->beam != GPUMCD_BEAM_SQUARE) return false;
    if (!std::isfinite(s->center_cm[0]) || !std::isfinite(s->center_cm[1])) return false;
    if (s->beam == GPUMCD_BEAM_SQUARE && !(s->field_cm >= 0.0 && std::isfinite(s->field_cm))) return false;
    if (s->n_spectrum < 0 || s->n_spectrum > GPUMCD_MAX_SPECTRUM_BINS) return false;
    if (s->n_spectrum == 0) return s->energy_mev > 0.0 && s->energy_mev <= c->phys.e_max;
    if (!s->spectrum_edges || !s->spectrum_weights) return false;
    double tot = 0.0;
    for (int i = 0; i < s->n_spectrum; ++i) {
        if (!(s->spectrum_edges[i + 1] > s->spectrum_edges[i])) return false;
        if (!(s->spectrum_weights[i] >= 0.0)) return false;
        tot += s->spectrum_weights[i];
    }
    return tot > 0.0 && s->spectrum_edges[0] > 0.0 && s->spectrum_edges[s->n_spectrum] <= c->phys.e_max;
}

gpumcd_status ensure_slot(gpumcd_ctx *c, Slot &sl, int grid, int block) {
    const size_t warps = (size_t)grid * (block / 32);
    ST(dev_alloc(c, sl.stacks, warps * NT * c->launch.stack_capacity * sizeof(Rec)));
    ST(dev_alloc(c, sl.hard, warps * HARD_CAP * sizeof(HardRec)));
    for (int b = 0; b < 2; ++b)
        for (int t = 0; t < NT; ++t)
            ST(dev_alloc(c, sl.queue[b][t], (size_t)c->launch.overflow_capacity * sizeof(Rec)));
    ST(dev_alloc(c, sl.control, sizeof(Control)));
    ST(dev_alloc(c, sl.plandev, sizeof(PlanDev) * GPUMCD_MAX_PLANS_PER_RUN));
    if (!sl.h_control) CK(cudaMallocHost(&sl.h_control, sizeof(Control)));
    if (!sl.h_plandev) CK(cudaMallocHost(&sl.h_plandev, sizeof(PlanDev) * GPUMCD_MAX_PLANS_PER_RUN));
    if (!sl.ev0) CK(cudaEventCreate(&sl.ev0));
    if (!sl.ev1) CK(cudaEventCreate(&sl.ev1));
    if (!sl.done) CK(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
    if (!c->configured) {
        CK(transport_configure());
        c->configured = true;
    }
    return GPUMCD_OK;
}

void free_slot(gpumcd_ctx *c, Slot &sl) {
    if (sl.busy && sl.s) cudaStreamSynchronize(sl.s);
    dev_free(c, sl.order);
    dev_free(c, sl.gcount);
    dev_free(c, sl.stacks);
    dev_free(c, sl.hard);
    for (int b = 0; b < 2; ++b)
        for (int t = 0; t < NT; ++t) dev_free(c, sl.queue[b][t]);
    dev_free(c, sl.control);
    dev_free(c, sl.plandev);
    if (sl.h_control) cudaFreeHost(sl.h_control);
    if (sl.h_plandev) cudaFreeHost(sl.h_plandev);
    if (sl.ev0) cudaEventDestroy(sl.ev0);
    if (sl.ev1) cudaEventDestroy(sl.ev1);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.gexec) cudaGraphExecDestroy(sl.gexec);
    if (sl.graph) cudaGraphDestroy(sl.graph);
    if (sl.own) cudaStreamDestroy(sl.own);
    sl = Slot{};
}

bool any_busy(const gpumcd_ctx *c) {
    for (const Slot &sl : c->slot)
        if (sl.busy) return true;
    return false;
}

}  // namespace

namespace gm {
Grid make_grid(const TableGeom &g) {
    const double ln2 = std::log(2.0), lq = std::log(kQ);
    const double dp = (std::log(g.p1) - std::log(g.p0)) / (G - 1);
    const double de = (std::log(g.e1) - std::log(g.e0)) / (G - 1);
    const double dm = (std::log(MS_G_MAX) - std::log(MS_G_MIN)) / (G_MS - 1);
    Grid r;
    r.ph_a = (float)(ln2 / dp);
    r.ph_bq = (float)((lq - std::log(g.p0)) / dp);
    r.el_a = (float)(ln2 / de);
    r.el_bq = (float)((lq - std::log(g.e0)) / de);
    r.el_bm = (float)(-std::log(g.e0) / de);
    r.ms_a = (float)(ln2 / dm);
    r.ms_b = (float)(-std::log(MS_G_MIN) / dm);
    return r;
}
}  // namespace gm

extern "C" {

const char *gpumcd_status_string(gpumcd_status s) {
    switch (s) {
        case GPUMCD_OK: return "ok";
        case GPUMCD_ERR_INVALID_ARG: return "invalid argument";
        case GPUMCD_ERR_OOM: return "device out of memory";
        case GPUMCD_ERR_CUDA: return "CUDA error";
        case GPUMCD_ERR_QUEUE_OVERFLOW: return "particle queue overflow";
        case GPUMCD_ERR_TIMEOUT: return "device wait timed out";
        case GPUMCD_ERR_NOT_FOUND: return "unknown id";
        case GPUMCD_ERR_BUDGET: return "HBM budget exceeded";
        case GPUMCD_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

gpumcd_status gpumcd_init(gpumcd_ctx **out, int32_t device, uint64_t hbm_budget_bytes) {
    if (!out) return GPUMCD_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return GPUMCD_ERR_CUDA;
    }
    if (device < 0 || device >= n) return GPUMCD_ERR_INVALID_ARG;
    gpumcd_ctx *c = new gpumcd_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
    size_t mem_free = 0, mem_total = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&mem_free, &mem_total);
    if (e == cudaSuccess) c->cache_max = std::max<uint64_t>(c->cache_max, mem_total / 2);
    // The context stream (tables, phantoms, folds, gpumcd_run by default) has
    // the highest priority, so a fold takes SMs first as a submitted
    // transport sequence drains; submitted sequences run at the lowest.
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->stream, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->order, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        delete c;
        return cuda_status(e);
    }
    c->launch.block_threads = 1024;
    c->launch.blocks_per_sm = 1;
    c->launch.stack_capacity = 512;
    c->launch.switch_high = 320;
    c->launch.refill_low = 16;
    c->launch.chunk = 32;
    c->launch.overflow_capacity = 1u << 20;
    c->launch.flags = 0;
    c->launch.refill_period = 1;
    *out = c;
    return GPUMCD_OK;
}

gpumcd_status gpumcd_destroy(gpumcd_ctx *c) {
    if (!c) return GPUMCD_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (Slot &sl : c->slot)
        if (sl.busy && sl.s) cudaStreamSynchronize(sl.s);
    for (auto &kv : c->plans) {
        if (kv.second.reset_done) cudaEventDestroy(kv.second.reset_done);
        dev_free(c, kv.second.tally);
        dev_free(c, kv.second.ledger);
        dev_free(c, kv.second.spec);
    }
    for (auto &kv : c->phantoms) {
        dev_free(c, kv.second.vox);
        dev_free(c, kv.second.rhomax);
        dev_free(c, kv.second.maj);
    }
    dev_free(c, c->tab);
    for (Slot &sl : c->slot) free_slot(c, sl);
    dev_free(c, c->fold_tmp);
    cache_trim(c, 0);
    if (c->order) cudaEventDestroy(c->order);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return GPUMCD_OK;
}

gpumcd_status gpumcd_load_materials(gpumcd_ctx *c, const gpumcd_material *mats, int32_t n,
                                    const gpumcd_physics *ph) {
    if (!c || !mats || !ph || n < 1 || n > GPUMCD_MAX_MATERIALS) return GPUMCD_ERR_INVALID_ARG;
    if (!c->phantoms.empty() || !c->plans.empty()) return GPUMCD_ERR_STATE;
    if (!(ph->p_cut > 0 && ph->e_abs > 0 && ph->t_c > 0 && ph->k_c > 0 && ph->estepe > 0 &&
          ph->estepe <= 1.0 && ph->e_max > ph->e_abs && ph->e_max > ph->p_cut && ph->e_max <= 20.0 &&
          ph->nudge_cm >= 0 && ph->nudge_cm < 1.0))
        return GPUMCD_ERR_INVALID_ARG;
    for (int m = 0; m < n; ++m) {
        const gpumcd_material &M = mats[m];
        if (M.n_elements < 1 || M.n_elements > GPUMCD_MAX_ELEMENTS || !(M.I_eV > 0)) return GPUMCD_ERR_INVALID_ARG;
        double ws = 0;
        for (int j = 0; j < M.n_elements; ++j) {
            if (M.Z[j] < 1 || M.Z[j] > 100 || !(M.A[j] > 0) || !(M.w[j] >= 0)) return GPUMCD_ERR_INVALID_ARG;
            ws += M.w[j];
        }
        if (!(ws > 0)) return GPUMCD_ERR_INVALID_ARG;
    }
    ST(set_device(c));
    ST(dev_alloc(c, c->tab, TAB_BYTES));
    c->phys = *ph;
    c->n_mat = n;
    c->geom.p0 = 0.5 * ph->p_cut;
    c->geom.p1 = ph->e_max * 1.0001;
    c->geom.e0 = 0.25 * std::fmin(ph->e_abs, ph->t_c);
    c->geom.e1 = ph->e_max * 1.0001;
    c->dphys.p_cut_q = (uint32_t)std::llround(ph->p_cut / kQ);
    c->dphys.e_abs_q = (uint32_t)std::llround(ph->e_abs / kQ);
    c->dphys.two_mc2_q = (uint32_t)std::llround(2.0 * kMC2 / kQ);
    c->dphys.t_c = (float)ph->t_c;
    c->dphys.k_c = (float)ph->k_c;
    c->dphys.estepe = (float)ph->estepe;
    c->dphys.nudge = (float)ph->nudge_cm;
    c->dphys.grid = make_grid(c->geom);
    CK(cudaMemsetAsync(c->tab.p, 0, TAB_BYTES, c->stream));
    CK(launch_build_tables(mats, n, c->geom, ph->t_c, ph->k_c, (float *)c->tab.p, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->tables = true;
    return GPUMCD_OK;
}

static gpumcd_status create_phantom_impl(gpumcd_ctx *c, const int32_t dims[3], const double voxel[3],
                                         const uint8_t *mat, const float *rho, bool device,
                                         cudaStream_t s, int32_t *id) {
    if (!c || !dims || !voxel || !mat || !rho || !id) return GPUMCD_ERR_INVALID_ARG;
    if (!c->tables) return GPUMCD_ERR_STATE;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || dims[a] > 4096) return GPUMCD_ERR_INVALID_ARG;
        if (!(voxel[a] > 0.0) || !std::isfinite(voxel[a])) return GPUMCD_ERR_INVALID_ARG;
    }
    const uint64_t nvox = (uint64_t)dims[0] * dims[1] * dims[2];
    if (nvox >= (1ull << 32)) return GPUMCD_ERR_INVALID_ARG;
    ST(set_device(c));
    Phantom ph{};
    for (int a = 0; a < 3; ++a) {
        ph.dims[a] = dims[a];
        ph.voxel[a] = voxel[a];
    }
    ph.nvox = nvox;
    gpumcd_status st = dev_alloc(c, ph.vox, nvox * 4);
    if (st == GPUMCD_OK) st = dev_alloc(c, ph.rhomax, 16 * 4);
    if (st == GPUMCD_OK) st = dev_alloc(c, ph.maj, MAJ_FLOATS * 4);
    DevBuf tmp_mat, tmp_rho, bad;
    if (st == GPUMCD_OK && !device) st = dev_alloc(c, tmp_mat, nvox);
    if (st == GPUMCD_OK && !device) st = dev_alloc(c, tmp_rho, nvox * 4);
    if (st == GPUMCD_OK) st = dev_alloc(c, bad, 4);
    cudaError_t e = cudaSuccess;
    int h_bad = 0;
    if (st == GPUMCD_OK) {
        const uint8_t *dm = mat;
        const float *dr = rho;
        if (!device) {
            e = cudaMemcpyAsync(tmp_mat.p, mat, nvox, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(tmp_rho.p, rho, nvox * 4, cudaMemcpyHostToDevice, s);
            dm = (const uint8_t *)tmp_mat.p;
            dr = (const float *)tmp_rho.p;
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(ph.rhomax.p, 0, 16 * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(bad.p, 0, 4, s);
        if (e == cudaSuccess)
            e = launch_pack_phantom(dm, dr, nvox, c->n_mat, (uint32_t *)ph.vox.p, (unsigned int *)ph.rhomax.p,
                                    (int *)bad.p, s);
        if (e == cudaSuccess)
            e = launch_majorants((const float *)c->tab.p, (const unsigned int *)ph.rhomax.p, c->n_mat,
                                 (float *)ph.maj.p, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad.p, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_status(e);
        else if (h_bad) st = GPUMCD_ERR_INVALID_ARG;
    }
    dev_free(c, tmp_mat);
    dev_free(c, tmp_rho);
    dev_free(c, bad);
    if (st != GPUMCD_OK) {
        dev_free(c, ph.vox);
        dev_free(c, ph.rhomax);
        dev_free(c, ph.maj);
        return st;
    }
    *id = c->next_id++;
    c->phantoms[*id] = ph;
    return GPUMCD_OK;
}

gpumcd_status gpumcd_create_phantom(gpumcd_ctx *c, const int32_t dims[3], const double voxel_cm[3],
                                    const uint8_t *material_ids, const float *densities, int32_t *id) {
    if (!c) return GPUMCD_ERR_INVALID_ARG;
    return create_phantom_impl(c, dims, voxel_cm, material_ids, densities, false, c->stream, id);
}

gpumcd_status gpumcd_create_phantom_device(gpumcd_ctx *c, const int32_t dims[3], const double voxel_cm[3],
                                           const uint8_t *material_ids, const float *densities, void *stream,
                                           int32_t *id) {
    if (!c) return GPUMCD_ERR_INVALID_ARG;
    return create_phantom_impl(c, dims, voxel_cm, material_ids, densities, true, pick(c, stream), id);
}

gpumcd_status gpumcd_destroy_phantom(gpumcd_ctx *c, int32_t id) {
    if (!c) return GPUMCD_ERR_INVALID_ARG;
    auto it = c->phantoms.find(id);
    if (it == c->phantoms.end()) return GPUMCD_ERR_NOT_FOUND;
    for (auto &kv : c->plans)
        if (kv.second.phantom == id) return GPUMCD_ERR_STATE;
    ST(set_device(c));
    cudaStreamSynchronize(c->stream);
    dev_free(c, it->second.vox);
    dev_free(c, it->second.rhomax);
    dev_free(c, it->second.maj);
    c->phantoms.erase(it);
    return GPUMCD_OK;
}

gpumcd_status gpumcd_plan_open(gpumcd_ctx *c, int32_t phantom_id, const gpumcd_source *src, uint64_t seed,
                               uint32_t n_batches, int32_t *plan_id) {
    if (!c || !plan_id) return GPUMCD_ERR_INVALID_ARG;
    if (!c->tables) return GPUMCD_ERR_STATE;
    auto it = c->phantoms.find(phantom_id);
    if (it == c->phantoms.end()) return GPUMCD_ERR_NOT_FOUND;
    if (!valid_source(c, src)) return GPUMCD_ERR_INVALID_ARG;
    if (n_batches == 0) n_batches = 32;
    if (n_batches < 8 || n_batches > 64 || (n_batches & (n_batches - 1))) return GPUMCD_ERR_INVALID_ARG;
    ST(set_device(c));
    Plan p{};
    p.phantom = phantom_id;
    p.particle = src->particle;
    p.beam = src->beam;
    p.energy = src->energy_mev;
    p.cx = src->center_cm[0];
    p.cy = src->center_cm[1];
    p.field = src->field_cm;
    p.n_spec = src->n_spectrum;
    p.e_group = (src->beam == GPUMCD_BEAM_PHASE_SPACE || src->n_spectrum > 0) &&
                src->energy_grouping == GPUMCD_ENERGY_GROUPED;
    p.seed = seed;
    p.W = n_batches;
    const uint64_t nvox = it->second.nvox;
    gpumcd_status st = dev_alloc(c, p.tally, (size_t)n_batches * nvox * 8);
    if (st == GPUMCD_OK) st = dev_alloc(c, p.ledger, 4 * 8);
    DevBuf tmp;
    if (st == GPUMCD_OK && p.n_spec > 0) {
        st = dev_alloc(c, p.spec, (size_t)2 * (p.n_spec + 1) * 4);
        if (st == GPUMCD_OK) st = dev_alloc(c, tmp, (size_t)(2 * p.n_spec + 1) * 8);
        if (st == GPUMCD_OK) {
            double *d = (double *)tmp.p;
            cudaError_t e = cudaMemcpyAsync(d, src->spectrum_edges, (p.n_spec + 1) * 8, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d + p.n_spec + 1, src->spectrum_weights, p.n_spec * 8, cudaMemcpyHostToDevice,
                                    c->stream);
            if (e == cudaSuccess) e = launch_spectrum(d, d + p.n_spec + 1, p.n_spec, (float *)p.spec.p, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) st = cuda_status(e);
        }
    }
    dev_free(c, tmp);
    if (st == GPUMCD_OK && p.beam == GPUMCD_BEAM_PHASE_SPACE) {
        // records as float4 pairs (x, y, z, E) (ux, uy, uz, 0), direction normalised,
        // in the listed order (energy grouping orders a launch's claims, not the list)
        const int32_t n = src->n_phase_space;
        for (int32_t i = 0; i < n; ++i) {
            const double *r = src->phase_space + 7 * (size_t)i;
            bool ok = true;
            for (int a = 0; a < 7; ++a) ok = ok && std::isfinite(r[a]);
            const double nu = std::sqrt(r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
            if (!ok || !(nu > 0.0) || !(r[6] > 0.0 && r[6] <= c->phys.e_max)) {
                st = GPUMCD_ERR_INVALID_ARG;
                break;
            }
        }
        std::vector<float> h((size_t)n * 8);
        for (int32_t i = 0; i < n && st == GPUMCD_OK; ++i) {
            const double *r = src->phase_space + 7 * (size_t)i;
            const double nu = std::sqrt(r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
            float *o = h.data() + 8 * (size_t)i;
            o[0] = (float)r[0], o[1] = (float)r[1], o[2] = (float)r[2], o[3] = (float)r[6];
            o[4] = (float)(r[3] / nu), o[5] = (float)(r[4] / nu), o[6] = (float)(r[5] / nu), o[7] = 0.f;
        }
        if (st == GPUMCD_OK) st = dev_alloc(c, p.spec, h.size() * sizeof(float));
        if (st == GPUMCD_OK) {
            cudaError_t e = cudaMemcpyAsync(p.spec.p, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice,
                                            c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) st = cuda_status(e);
        }
        p.n_phsp = (uint32_t)n;
        p.n_spec = 0;
    }
    if (st == GPUMCD_OK) {
        cudaError_t e = cudaMemsetAsync(p.tally.p, 0, (size_t)n_batches * nvox * 8, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(p.ledger.p, 0, 4 * 8, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = cuda_status(e);
    }
    if (st != GPUMCD_OK) {
        dev_free(c, p.tally);
        dev_free(c, p.ledger);
        dev_free(c, p.spec);
        return st;
    }
    if (cudaEventCreateWithFlags(&p.reset_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        dev_free(c, p.tally);
        dev_free(c, p.ledger);
        dev_free(c, p.spec);
        return GPUMCD_ERR_CUDA;
    }
    *plan_id = c->next_id++;
    c->plans[*plan_id] = p;
    return GPUMCD_OK;
}

gpumcd_status gpumcd_plan_close(gpumcd_ctx *c, int32_t plan_id) {
    if (!c) return GPUMCD_ERR_INVALID_ARG;
    auto it = c->plans.find(plan_id);
    if (it == c->plans.end()) return GPUMCD_ERR_NOT_FOUND;
    if (it->second.inflight > 0) return GPUMCD_ERR_STATE;
    ST(set_device(c));
    // the tally goes back to the cache: wait for the context stream and for
    // the last reset's memsets, which may have run on a caller's stream
    cudaStreamSynchronize(c->stream);
    if (it->second.reset_done) {
        cudaEventSynchronize(it->second.reset_done);
        cudaEventDestroy(it->second.reset_done);
    }
    dev_free(c, it->second.tally);
    dev_free(c, it->second.ledger);
    dev_free(c, it->second.spec);
    c->plans.erase(it);
    return GPUMCD_OK;
}

gpumcd_status gpumcd_plan_reset(gpumcd_ctx *c, int32_t plan_id, uint64_t seed, void *stream) {
    if (!c) return GPUMCD_ERR_INVALID_ARG;
    auto it = c->plans.find(plan_id);
    if (it == c->plans.end()) return GPUMCD_ERR_NOT_FOUND;
    if (it->second.inflight > 0) return GPUMCD_ERR_STATE;
    ST(set_device(c));
    cudaStream_t s = pick(c, stream);
    Plan &p = it->second;
    // a cached block may be larger than the tally: zero the tally's own size
    CK(cudaMemsetAsync(p.tally.p, 0, (size_t)p.W * c->phantoms.at(p.phantom).nvox * 8, s));
    CK(cudaMemsetAsync(p.ledger.p, 0, 4 * 8, s));
    CK(cudaEventRecord(p.reset_done, s));
    p.seed = seed;
    p.hist_sub = 0;
    p.hist_done = 0;
    p.failed = false;
    p.acc = gpumcd_run_stats{};
    return GPUMCD_OK;
}

gpumcd_status gpumcd_plan_histories(gpumcd_ctx *c, int32_t plan_id, uint64_t *h) {
    if (!c || !h) return GPUMCD_ERR_INVALID_ARG;
    auto it = c->plans.find(plan_id);
    if (it == c->plans.end()) return GPUMCD_ERR_NOT_FOUND;
    *h = it->second.hist_done;
    return GPUMCD_OK;
}

}  // extern "C"

namespace {

// Enqueue launch k of a sequence: the in-queue is the previous launch's
// out-queue (empty for k = 0), both cursors restart at 0.
gpumcd_status launch_one(gpumcd_ctx *c, Slot &sl) {
    const int bi = (int)(sl.k & 1u), bo = bi ^ 1;
    Control *dc = (Control *)sl.control.p;
    TransportArgs &A = sl.A;
    for (int t = 0; t < NT; ++t) {
        A.in[t].rec = (Rec *)sl.queue[bi][t].p;
        A.in[t].cursor = &dc->qcur[bi][t];
        A.in[t].capacity = c->launch.overflow_capacity;
        A.out[t].rec = (Rec *)sl.queue[bo][t].p;
        A.out[t].cursor = &dc->qcur[bo][t];
        A.out[t].capacity = c->launch.overflow_capacity;
        A.in_count[t] = sl.in_count[t];
    }
    CK(cudaMemsetAsync(dc->qcur, 0, sizeof(dc->qcur), sl.s));
    CK(launch_transport(A, sl.grid, sl.block, sl.bps, sl.s));
    CK(cudaMemcpyAsync(sl.h_control, dc, sizeof(Control), cudaMemcpyDeviceToHost, sl.s));
    CK(cudaEventRecord(sl.done, sl.s));
    ++sl.k;
    return GPUMCD_OK;
}

// The queue and cursor pointers of launch k = 0 (empty in-queue).
void first_queues(gpumcd_ctx *c, Slot &sl) {
    Control *dc = (Control *)sl.control.p;
    for (int t = 0; t < NT; ++t) {
        sl.A.in[t].rec = (Rec *)sl.queue[0][t].p;
        sl.A.in[t].cursor = &dc->qcur[0][t];
        sl.A.in[t].capacity = c->launch.overflow_capacity;
        sl.A.out[t].rec = (Rec *)sl.queue[1][t].p;
        sl.A.out[t].cursor = &dc->qcur[1][t];
        sl.A.out[t].capacity = c->launch.overflow_capacity;
        sl.A.in_count[t] = 0;
    }
}

// First launch of a sequence from the slot's captured graph.  Its copy and
// reset nodes touch only slot-owned buffers of fixed size (the whole plan
// table is copied), so the graph stays valid for the slot's lifetime and
// only the kernel node's argument block changes between runs; a new launch
// shape (grid, CTA size, kernel variant) is captured afresh.
gpumcd_status first_launch_graph(gpumcd_ctx *c, Slot &sl) {
    first_queues(c, sl);
    Control *dc = (Control *)sl.control.p;
    // a graph is rebuilt for a new launch shape or another compiled kernel
    // (its kernel node keeps the function it was captured with)
    const void *fn = transport_kernel(sl.A, sl.block, sl.bps);
    if (!sl.gexec || sl.g_grid != sl.grid || sl.g_block != sl.block || sl.g_bps != sl.bps || sl.g_fn != fn) {
        if (sl.gexec) cudaGraphExecDestroy(sl.gexec);
        if (sl.graph) cudaGraphDestroy(sl.graph);
        sl.gexec = nullptr;
        sl.graph = nullptr;
        sl.knode = nullptr;
        CK(cudaStreamBeginCapture(sl.s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemcpyAsync(sl.plandev.p, sl.h_plandev, sizeof(PlanDev) * GPUMCD_MAX_PLANS_PER_RUN,
                                        cudaMemcpyHostToDevice, sl.s);
        if (e == cudaSuccess) e = cudaMemsetAsync(dc, 0, sizeof(Control), sl.s);
        if (e == cudaSuccess) e = launch_transport(sl.A, sl.grid, sl.block, sl.bps, sl.s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_control, dc, sizeof(Control), cudaMemcpyDeviceToHost, sl.s);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(sl.s, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&sl.gexec, g, 0);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            sl.gexec = nullptr;
            return cuda_status(e);
        }
        sl.graph = g;
        size_t n = 0;
        CK(cudaGraphGetNodes(g, nullptr, &n));
        std::vector<cudaGraphNode_t> nodes(n);
        CK(cudaGraphGetNodes(g, nodes.data(), &n));
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType ty;
            CK(cudaGraphNodeGetType(nd, &ty));
            if (ty == cudaGraphNodeTypeKernel) sl.knode = nd;
        }
        if (!sl.knode) return GPUMCD_ERR_CUDA;
        sl.g_grid = sl.grid;
        sl.g_block = sl.block;
        sl.g_bps = sl.bps;
        sl.g_fn = fn;
    } else {
        cudaKernelNodeParams kp;
        CK(cudaGraphKernelNodeGetParams(sl.knode, &kp));
        void *args[] = {&sl.A};
        kp.kernelParams = args;
        kp.extra = nullptr;
        CK(cudaGraphExecKernelNodeSetParams(sl.gexec, sl.knode, &kp));
    }
    CK(cudaEventRecord(sl.ev0, sl.s));
    CK(cudaGraphLaunch(sl.gexec, sl.s));
    CK(cudaEventRecord(sl.done, sl.s));
    sl.k = 1;
    return GPUMCD_OK;
}

// Settle a sequence: per-plan accounting, then the slot is free again.
void seq_close(gpumcd_ctx *c, Slot &sl, gpumcd_status result, float ms) {
    for (size_t i = 0; i < sl.ids.size(); ++i) {
        auto it = c->plans.find(sl.ids[i]);
        if (it == c->plans.end()) continue;
        Plan &p = it->second;
        --p.inflight;
        if (result == GPUMCD_OK) p.hist_done += sl.n_hist[i];
        else p.failed = true;
        p.acc.n_launches += sl.k;
        p.acc.transport_ms += ms;
    }
    if (result == GPUMCD_OK || sl.k > 0) {
        c->last = *sl.h_control;
        c->have_last = true;
        // run-wide counters go to every plan of a single-plan run and to the first plan otherwise
        auto it = c->plans.find(sl.ids[0]);
        if (it != c->plans.end()) {
            gpumcd_run_stats &a = it->second.acc;
            const unsigned long long *n = c->last.counters;
            a.n_photon_events += n[CNT_PH_EVENTS];
            a.n_photon_real += n[CNT_PH_REAL];
            a.n_compton += n[CNT_COMPTON];
            a.n_photo += n[CNT_PHOTO];
            a.n_pair += n[CNT_PAIR];
            a.n_electron_steps += n[CNT_E_STEPS];
            a.n_hard_real += n[CNT_HARD_REAL];
            a.n_hard_fict += n[CNT_HARD_FICT];
            a.n_moller += n[CNT_MOLLER];
            a.n_brem += n[CNT_BREM];
            a.n_photons += n[CNT_PHOTONS];
            a.n_electrons += n[CNT_ELECTRONS];
            a.n_overflow += n[CNT_OVERFLOW];
            a.n_spilled += n[CNT_SPILLS];
            a.n_sampler_capped += n[CNT_SAMPLER_CAP];
        }
    }
    sl.busy = false;
    sl.ticket = 0;
    sl.ids.clear();
    sl.n_hist.clear();
}

// Validate a run request and enqueue its first launch on stream s.
// Histories of a grouped source a launch sorts by energy at most (2^28, a
// 1 GB claim order); the rest of a larger run is claimed as numbered.
constexpr uint64_t kGroupSortMax = 1ull << 28;

gpumcd_status seq_start(gpumcd_ctx *c, Slot &sl, int32_t n_plans, const int32_t *ids, const uint64_t *n_hist,
                        cudaStream_t s) {
    if (n_plans < 1 || n_plans > GPUMCD_MAX_PLANS_PER_RUN || !ids || !n_hist) return GPUMCD_ERR_INVALID_ARG;
    if (!c->tables) return GPUMCD_ERR_STATE;
    std::vector<Plan *> pl(n_plans);
    for (int i = 0; i < n_plans; ++i) {
        auto it = c->plans.find(ids[i]);
        if (it == c->plans.end()) return GPUMCD_ERR_NOT_FOUND;
        for (int j = 0; j < i; ++j)
            if (ids[j] == ids[i]) return GPUMCD_ERR_INVALID_ARG;
        pl[i] = &it->second;
        if (pl[i]->failed) return GPUMCD_ERR_STATE;
        if (pl[i]->hist_sub + n_hist[i] > (1ull << 32)) return GPUMCD_ERR_INVALID_ARG;
    }
    ST(set_device(c));
    sl.block = (int)c->launch.block_threads;
    sl.bps = (int)c->launch.blocks_per_sm;
    sl.grid = c->n_sm * sl.bps;
    ST(ensure_slot(c, sl, sl.grid, sl.block));

    TransportArgs &A = sl.A;
    memset(&A, 0, sizeof A);
    for (int i = 0; i < n_plans; ++i) {
        const Plan &p = *pl[i];
        const Phantom &ph = c->phantoms.at(p.phantom);
        PlanDev &d = sl.h_plandev[i];
        memset(&d, 0, sizeof d);
        d.vox = (const uint32_t *)ph.vox.p;
        d.tally = (unsigned long long *)p.tally.p;
        d.ledger = (unsigned long long *)p.ledger.p;
        d.maj = (const float *)ph.maj.p;
        d.spec = (const float *)p.spec.p;
        d.nx = ph.dims[0];
        d.ny = ph.dims[1];
        d.nz = ph.dims[2];
        d.n_spec = p.n_spec;
        d.dx = (float)ph.voxel[0];
        d.dy = (float)ph.voxel[1];
        d.dz = (float)ph.voxel[2];
        d.inv_dx = (float)(1.0 / ph.voxel[0]);
        d.inv_dy = (float)(1.0 / ph.voxel[1]);
        d.inv_dz = (float)(1.0 / ph.voxel[2]);
        d.X = (float)(ph.dims[0] * ph.voxel[0]);
        d.Y = (float)(ph.dims[1] * ph.voxel[1]);
        d.Z = (float)(ph.dims[2] * ph.voxel[2]);
        d.cx = (float)p.cx;
        d.cy = (float)p.cy;
        d.field = (float)p.field;
        d.nvox = (uint32_t)ph.nvox;
        d.bmask = p.W - 1;
        d.key_lo = (uint32_t)p.seed;
        d.key_hi = (uint32_t)(p.seed >> 32);
        d.src_type = p.particle;
        d.beam = p.beam;
        d.e_src_q = (uint32_t)std::llround(p.energy / kQ);
        d.n_phsp = p.n_phsp;
        d.e_group = p.e_group ? 1u : 0u;
        if (p.n_phsp || p.e_group) A.phsp = 1;
        d.hist_base = p.hist_sub;
        if (p.e_group) d.n_sorted = (uint32_t)std::min<uint64_t>(n_hist[i], kGroupSortMax);
        const int t = p.particle;
        A.prim_plan[t][A.n_prim_plans[t]] = (uint8_t)i;
        A.prim_off[t][A.n_prim_plans[t] + 1] = A.prim_off[t][A.n_prim_plans[t]] + n_hist[i];
        A.n_prim_plans[t]++;
    }
    Control *dc = (Control *)sl.control.p;
    A.tables = (const float *)c->tab.p;
    A.tab_bytes = tab_bytes(c->n_mat);
    A.phys = c->dphys;
    A.plans = (const PlanDev *)sl.plandev.p;
    A.n_plans = n_plans;
    A.prim_cursor = dc->prim_cursor;
    A.stacks = (Rec *)sl.stacks.p;
    A.hard = (HardRec *)sl.hard.p;
    A.stack_cap = c->launch.stack_capacity;
    A.switch_high = c->launch.switch_high;
    A.refill_low = c->launch.refill_low;
    A.refill_period = c->launch.refill_period;
    // the phase-space kernel is its own instantiation, without the other special ones
    if (A.phsp && (c->launch.refill_period != 1u ||
                   (c->launch.flags & (GPUMCD_LAUNCH_PROFILE | GPUMCD_LAUNCH_WARP_AGGREGATE | GPUMCD_LAUNCH_KERMA))))
        return GPUMCD_ERR_INVALID_ARG;
    A.chunk = c->launch.chunk;
    A.flags = c->launch.flags;
    A.counters = dc->counters;
    A.error = &dc->error;

    // sources grouped by energy: sort each one's histories of this launch by
    // energy, on the sequence's stream ahead of the launch
    // (the orders of all grouped plans, then one plan's keys: the plans' sorts
    // run one after another on the stream and share the key scratch)
    size_t n_order = 0, n_keys = 0;
    for (int i = 0; i < n_plans; ++i) {
        const PlanDev &d = sl.h_plandev[i];
        if (!d.e_group) continue;
        n_order += d.n_sorted;
        n_keys = std::max<size_t>(n_keys, d.n_sorted);
    }
    if (n_order > 0) {
        const size_t bytes = n_order * 4 + n_keys * 2;
        if (sl.order.bytes < bytes) {
            dev_free(c, sl.order);  // the slot's last sequence has finished: nothing pending on it
            ST(dev_alloc(c, sl.order, bytes));
        }
        if (!sl.gcount.p) ST(dev_alloc(c, sl.gcount, GPUMCD_MAX_SPECTRUM_BINS * sizeof(unsigned)));
        uint32_t *ord = (uint32_t *)sl.order.p;
        uint16_t *keys = (uint16_t *)((uint32_t *)sl.order.p + n_order);
        for (int i = 0; i < n_plans; ++i) {
            PlanDev &d = sl.h_plandev[i];
            if (!d.e_group) continue;
            d.order = ord;
            CK(launch_group_order(d, d.n_sorted, (unsigned *)sl.gcount.p, keys, ord, s));
            ord += d.n_sorted;
        }
    }

    sl.s = s;
    sl.k = 0;
    sl.in_count[0] = sl.in_count[1] = 0;
    sl.ids.assign(ids, ids + n_plans);
    sl.n_hist.assign(n_hist, n_hist + n_plans);
    sl.busy = true;
    for (int i = 0; i < n_plans; ++i) {
        pl[i]->hist_sub += n_hist[i];
        ++pl[i]->inflight;
    }
    gpumcd_status st = GPUMCD_OK;
    if (c->launch.flags & GPUMCD_LAUNCH_GRAPH) {
        st = first_launch_graph(c, sl);
    } else {
        cudaError_t e = cudaMemcpyAsync(sl.plandev.p, sl.h_plandev, sizeof(PlanDev) * n_plans,
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(dc, 0, sizeof(Control), s);
        if (e == cudaSuccess) e = cudaEventRecord(sl.ev0, s);
        st = cuda_status(e);
        if (st == GPUMCD_OK) st = launch_one(c, sl);
    }
    if (st != GPUMCD_OK) {
        if (sl.s) cudaStreamSynchronize(sl.s);
        seq_close(c, sl, st, 0.f);
    }
    return st;
}

// Wait for the sequence's last enqueued launch; relaunch over the overflow
// queues while they hold particles; then account and free the slot.
gpumcd_status seq_finish(gpumcd_ctx *c, Slot &sl) {
    gpumcd_status result = GPUMCD_OK;
    for (;;) {
        cudaError_t e = cudaEventSynchronize(sl.done);
        if (e != cudaSuccess) {
            result = cuda_status(e);
            break;
        }
        const Control &hc = *sl.h_control;
        if (hc.error != 0) {
            result = hc.error;
            break;
        }
        const int bo = (int)((sl.k - 1u) & 1u) ^ 1;
        bool more = false;
        for (int t = 0; t < NT; ++t) {
            const unsigned long long o = hc.qcur[bo][t];
            sl.in_count[t] = o < c->launch.overflow_capacity ? o : c->launch.overflow_capacity;
            more = more || o > 0;
        }
        if (!more) break;
        if (sl.k >= 1000) {
            result = GPUMCD_ERR_TIMEOUT;
            break;
        }
        result = launch_one(c, sl);
        if (result != GPUMCD_OK) break;
    }
    float ms = 0.f;
    if (cudaEventRecord(sl.ev1, sl.s) == cudaSuccess && cudaEventSynchronize(sl.ev1) == cudaSuccess)
        cudaEventElapsedTime(&ms, sl.ev0, sl.ev1);
    else
        cudaGetLastError();
    seq_close(c, sl, result, ms);
    return result;
}

Slot *find_ticket(gpumcd_ctx *c, int32_t ticket) {
    for (int i = 1; i <= GPUMCD_MAX_INFLIGHT; ++i)
        if (c->slot[i].busy && c->slot[i].ticket == ticket) return &c->slot[i];
    return nullptr;
}

}  // namespace

extern "C" {

gpumcd_status gpumcd_run(gpumcd_ctx *c, int32_t n_plans, const int32_t *ids, const uint64_t *n_hist, void *stream) {
    if (!c) return GPUMCD_ERR_INVALID_ARG;
    Slot &sl = c->slot[0];
    if (sl.busy) return GPUMCD_ERR_STATE;
    // A set holding both electron and photon plans runs as one sequence per
    // particle type, electrons first.  In one launch the warps would draw both
    // kinds of primaries at once and switch type far more often; on the C4
    // set that cost as much as batching saves (388 vs 375 ms).  The tallies do
    // not depend on the split.  The whole set is validated before anything
    // runs, so a rejected set runs nothing.
    if (n_plans > 1 && n_plans <= GPUMCD_MAX_PLANS_PER_RUN && ids && n_hist) {
        std::vector<int32_t> id_t[2];
        std::vector<uint64_t> n_t[2];
        bool ok = true;
        for (int i = 0; i < n_plans && ok; ++i) {
            auto it = c->plans.find(ids[i]);
            if (it == c->plans.end() || it->second.failed || it->second.hist_sub + n_hist[i] > (1ull << 32)) {
                ok = false;
                break;
            }
            for (int j = 0; j < i; ++j)
                if (ids[j] == ids[i]) ok = false;
            const int t = it->second.particle == GPUMCD_ELECTRON ? 0 : 1;
            id_t[t].push_back(ids[i]);
            n_t[t].push_back(n_hist[i]);
        }
        if (ok && !id_t[0].empty() && !id_t[1].empty()) {
            for (int t = 0; t < 2; ++t) {
                ST(seq_start(c, sl, (int32_t)id_t[t].size(), id_t[t].data(), n_t[t].data(), pick(c, stream)));
                ST(seq_finish(c, sl));
            }
            return GPUMCD_OK;
        }
    }
    ST(seq_start(c, sl, n_plans, ids, n_hist, pick(c, stream)));
    return seq_finish(c, sl);
}

gpumcd_status gpumcd_submit(gpumcd_ctx *c, int32_t n_plans, const int32_t *ids, const uint64_t *n_hist,
                            int32_t *ticket) {
    if (!c || !ticket) return GPUMCD_ERR_INVALID_ARG;
    *ticket = 0;
    Slot *sl = nullptr;
    for (int i = 1; i <= GPUMCD_MAX_INFLIGHT && !sl; ++i)
        if (!c->slot[i].busy) sl = &c->slot[i];
    if (!sl) return GPUMCD_ERR_STATE;
    ST(set_device(c));
    if (!sl->own) {
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CK(cudaStreamCreateWithPriority(&sl->own, cudaStreamNonBlocking, least));
    }
    // after everything already enqueued on the context stream (plan resets, phantoms)
    CK(cudaEventRecord(c->order, c->stream));
    CK(cudaStreamWaitEvent(sl->own, c->order, 0));
    ST(seq_start(c, *sl, n_plans, ids, n_hist, sl->own));
    sl->ticket = c->next_ticket++;
    if (c->next_ticket <= 0) c->next_ticket = 1;
    *ticket = sl->ticket;
    return GPUMCD_OK;
}

gpumcd_status gpumcd_poll(gpumcd_ctx *c, int32_t ticket, int32_t *done) {
    if (!c || !done) return GPUMCD_ERR_INVALID_ARG;
    *done = 0;
    Slot *sl = find_ticket(c, ticket);
    if (!sl) return GPUMCD_ERR_NOT_FOUND;
    ST(set_device(c));
    const cudaError_t e = cudaEventQuery(sl->done);
    if (e == cudaErrorNotReady) {
        cudaGetLastError();
        return GPUMCD_OK;
    }
    *done = 1;
    return seq_finish(c, *sl);
}

gpumcd_status gpumcd_wait(gpumcd_ctx *c, int32_t ticket) {
    if (!c) return GPUMCD_ERR_INVALID_ARG;
    Slot *sl = find_ticket(c, ticket);
    if (!sl) return GPUMCD_ERR_NOT_FOUND;
    ST(set_device(c));
    return seq_finish(c, *sl);
}

gpumcd_status gpumcd_plan_result(gpumcd_ctx *c, int32_t plan_id, double thr, double *dose, double *sigma,
                                 void *stream, gpumcd_run_stats *stats) {
    if (!c) return GPUMCD_ERR_INVALID_ARG;
    auto it = c->plans.find(plan_id);
    if (it == c->plans.end()) return GPUMCD_ERR_NOT_FOUND;
    if (!(thr >= 0.0 && thr <= 1.0)) return GPUMCD_ERR_INVALID_ARG;
    if (it->second.inflight > 0 || it->second.failed) return GPUMCD_ERR_STATE;
    ST(set_device(c));
    cudaStream_t s = pick(c, stream);
    Plan &p = it->second;
    const Phantom &ph = c->phantoms.at(p.phantom);
    const uint64_t nvox = ph.nvox;
    // scratch: [dose | sigma] when the caller passes NULL, then [n_b (64) | dmax | sum | count | esum],
    // then the s_thr reduction's per-block partials
    const size_t need = (size_t)nvox * 16 + 64 * 8 + 64 + (size_t)sthr_blocks(nvox, c->n_sm) * 16;
    ST(dev_alloc(c, c->fold_tmp, need));
    double *tdose = (double *)c->fold_tmp.p;
    double *tsig = tdose + nvox;
    double *nb = tsig + nvox;
    unsigned long long *red = (unsigned long long *)(nb + 64);
    void *sthr_part = red + 8;
    double *ddose = dose ? dose : tdose;
    double *dsig = sigma ? sigma : tsig;
    double h_nb[64] = {0};
    const uint64_t N = p.hist_done;
    // history h belongs to batch h mod W
    for (uint32_t b = 0; b < p.W; ++b) h_nb[b] = (double)(N / p.W + (b < N % p.W ? 1u : 0u));
    CK(cudaMemsetAsync(red, 0, 64, s));
    const double inv_vol = 1.0 / (ph.voxel[0] * ph.voxel[1] * ph.voxel[2]);
    if (N > 0) {
        CK(launch_fold((const unsigned long long *)p.tally.p, (const uint32_t *)ph.vox.p, nvox, (int)p.W, h_nb,
                       (double)N, inv_vol, ddose, dsig, red, red + 3, c->n_sm, s));
        CK(launch_sthr(ddose, dsig, nvox, red, thr, (double *)(red + 1), red + 2, sthr_part, c->n_sm, s));
    } else {
        CK(cudaMemsetAsync(ddose, 0, nvox * 8, s));
        CK(cudaMemsetAsync(dsig, 0, nvox * 8, s));
    }
    unsigned long long h_red[4], h_led[4];
    CK(cudaMemcpyAsync(h_red, red, sizeof h_red, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h_led, p.ledger.p, sizeof h_led, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (stats) {
        *stats = p.acc;
        stats->histories = N;
        stats->n_batches = p.W;
        stats->e_incident = h_led[0];
        stats->e_escaped = h_led[1];
        stats->e_rest = h_led[2];
        stats->e_deposited = h_red[3];
        double dm;
        memcpy(&dm, &h_red[0], 8);
        stats->d_max_gy = dm;
        double ssum;
        memcpy(&ssum, &h_red[1], 8);
        stats->s_thr = h_red[2] ? ssum / (double)h_red[2] : 0.0;
    }
    return GPUMCD_OK;
}

gpumcd_status gpumcd_plan_result_noalloc(gpumcd_ctx *c, int32_t plan_id, double thr, double *dose, double *sigma,
                                         void *stream, gpumcd_run_stats *stats) {
    if (!c || !dose || !sigma) return GPUMCD_ERR_INVALID_ARG;
    auto it = c->plans.find(plan_id);
    if (it == c->plans.end()) return GPUMCD_ERR_NOT_FOUND;
    if (!(thr >= 0.0 && thr <= 1.0)) return GPUMCD_ERR_INVALID_ARG;
    Plan &p = it->second;
    if (p.inflight > 0 || p.failed) return GPUMCD_ERR_STATE;
    const Phantom &ph = c->phantoms.at(p.phantom);
    if (ph.nvox > (uint64_t)GPUMCD_NOALLOC_MAX_VOXELS) return GPUMCD_ERR_INVALID_ARG;
    const uint64_t N = p.hist_done;
    if (N == 0) return GPUMCD_ERR_STATE;
    ST(set_device(c));
    cudaStream_t s = pick(c, stream);
    double h_nb[64] = {0};
    // history h belongs to batch h mod W
    for (uint32_t b = 0; b < p.W; ++b) h_nb[b] = (double)(N / p.W + (b < N % p.W ? 1u : 0u));
    unsigned long long res[4] = {0, 0, 0, 0}, led[4] = {0, 0, 0, 0};
    const double inv_vol = 1.0 / (ph.voxel[0] * ph.voxel[1] * ph.voxel[2]);
    CK(launch_fold_noalloc(c->device, (const unsigned long long *)p.tally.p, (const uint32_t *)ph.vox.p, ph.nvox,
                           (int)p.W, h_nb, (double)N, inv_vol, thr, dose, sigma, s, res));
    CK(cudaMemcpyAsync(led, p.ledger.p, sizeof led, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (stats) {
        *stats = p.acc;
        stats->histories = N;
        stats->n_batches = p.W;
        stats->e_incident = led[0];
        stats->e_escaped = led[1];
        stats->e_rest = led[2];
        stats->e_deposited = res[1];
        memcpy(&stats->d_max_gy, &res[0], 8);
        memcpy(&stats->s_thr, &res[2], 8);
    }
    return GPUMCD_OK;
}

gpumcd_status gpumcd_plan_result_host(gpumcd_ctx *c, int32_t plan_id, double thr, double *dose, double *sigma,
                                      gpumcd_run_stats *stats) {
    if (!c) return GPUMCD_ERR_INVALID_ARG;
    auto it = c->plans.find(plan_id);
    if (it == c->plans.end()) return GPUMCD_ERR_NOT_FOUND;
    // the fold writes [dose | sigma] into the context's fold scratch, then both
    // arrays come back in two copies on the context's stream
    ST(gpumcd_plan_result(c, plan_id, thr, nullptr, nullptr, nullptr, stats));
    const uint64_t nvox = c->phantoms.at(it->second.phantom).nvox;
    const double *td = (const double *)c->fold_tmp.p;
    if (dose) CK(cudaMemcpyAsync(dose, td, nvox * 8, cudaMemcpyDeviceToHost, c->stream));
    if (sigma) CK(cudaMemcpyAsync(sigma, td + nvox, nvox * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return GPUMCD_OK;
}

// Rounds of at least this many histories run in a launch of their own in
// gpumcd_run_to_uncertainty (2^23).
constexpr uint64_t kAloneHistories = 1ull << 23;

gpumcd_status gpumcd_run_to_uncertainty(gpumcd_ctx *c, int32_t n_plans, const int32_t *ids,
                                        const uint64_t *first, const uint64_t *max_hist, double target,
                                        double thr, void *stream, uint64_t *hist_out, double *s_out,
                                        uint32_t *rounds_out, double *transport_ms_out, uint32_t *sequences_out) {
    if (!c || n_plans < 1 || n_plans > GPUMCD_MAX_PLANS_PER_RUN || !ids || !first || !max_hist) return GPUMCD_ERR_INVALID_ARG;
    if (!(target > 0.0) || !(thr >= 0.0 && thr <= 1.0)) return GPUMCD_ERR_INVALID_ARG;
    std::vector<uint64_t> done(n_plans), goal(n_plans);
    std::vector<double> s(n_plans, INFINITY);
    std::vector<uint32_t> W(n_plans);
    for (int i = 0; i < n_plans; ++i) {
        auto it = c->plans.find(ids[i]);
        if (it == c->plans.end()) return GPUMCD_ERR_NOT_FOUND;
        for (int j = 0; j < i; ++j)
            if (ids[j] == ids[i]) return GPUMCD_ERR_INVALID_ARG;
        if (it->second.inflight > 0 || it->second.failed) return GPUMCD_ERR_STATE;
        if (first[i] < 1 || max_hist[i] < first[i] || max_hist[i] > (1ull << 32)) return GPUMCD_ERR_INVALID_ARG;
        done[i] = it->second.hist_done;
        W[i] = it->second.W;
        goal[i] = done[i] + first[i];
    }
    std::vector<char> active(n_plans, 1);
    uint32_t rounds = 0, sequences = 0;
    double transport_ms = 0.0;
    for (;;) {
        // this round: every active plan runs up to its goal, in whole multiples of
        // its W batches (so the batches stay equal), within its history cap
        std::vector<int32_t> rid;
        std::vector<uint64_t> rn;
        for (int i = 0; i < n_plans; ++i) {
            if (!active[i]) continue;
            const uint64_t diff = goal[i] > done[i] ? goal[i] - done[i] : 0;
            uint64_t n = std::max<uint64_t>(W[i], (diff + W[i] - 1) / W[i] * W[i]);
            n = std::min<uint64_t>(n, max_hist[i] - done[i]);
            if (n == 0) {
                active[i] = 0;
                continue;
            }
            rid.push_back(ids[i]);
            rn.push_back(n);
        }
        if (rid.empty()) break;
        // A plan whose round holds at least kAloneHistories runs in a launch of
        // its own; the others share one launch sequence per particle type.
        // Sharing saves the fixed cost of a launch (its drain, about half a
        // millisecond) but mixes the plans' phantoms and tallies in the SMs'
        // L1; for rounds this large the launch costs < 1% and the mix more.
        std::vector<int32_t> sid;
        std::vector<uint64_t> sn;
        for (size_t r = 0; r < rid.size(); ++r) {
            if (rn[r] >= kAloneHistories) {
                const double before = c->plans.at(rid[r]).acc.transport_ms;
                ST(gpumcd_run(c, 1, &rid[r], &rn[r], stream));
                transport_ms += c->plans.at(rid[r]).acc.transport_ms - before;
                ++sequences;
            } else {
                sid.push_back(rid[r]);
                sn.push_back(rn[r]);
            }
        }
        if (!sid.empty()) {
            // one sequence per particle type: its device time is the growth of
            // one plan's transport time per type
            double before[2] = {-1.0, -1.0};
            int32_t probe[2] = {-1, -1};
            for (int32_t id : sid) {
                const Plan &pl = c->plans.at(id);
                const int t = pl.particle == GPUMCD_ELECTRON ? 1 : 0;
                if (probe[t] < 0) {
                    probe[t] = id;
                    before[t] = pl.acc.transport_ms;
                }
            }
            ST(gpumcd_run(c, (int32_t)sid.size(), sid.data(), sn.data(), stream));
            for (int t = 0; t < 2; ++t)
                if (probe[t] >= 0) {
                    transport_ms += c->plans.at(probe[t]).acc.transport_ms - before[t];
                    ++sequences;
                }
        }
        ++rounds;
        for (size_t r = 0, i = 0; r < rid.size(); ++r) {
            while (ids[i] != rid[r]) ++i;
            done[i] += rn[r];
            gpumcd_run_stats st{};
            ST(gpumcd_plan_result(c, ids[i], thr, nullptr, nullptr, stream, &st));
            s[i] = st.s_thr > 0.0 ? st.s_thr : INFINITY;
            if (s[i] <= target || done[i] >= max_hist[i]) {
                active[i] = 0;
            } else {
                // s falls as 1/sqrt(N): the count expected to reach the target,
                // with 5% to spare, and at least 10% more than now
                const double want = std::max((double)done[i] * (s[i] / target) * (s[i] / target) * 1.05,
                                             (double)done[i] * 1.1);
                goal[i] = want >= (double)max_hist[i] ? max_hist[i] : (uint64_t)want;
            }
        }
    }
    for (int i = 0; i < n_plans; ++i) {
        if (hist_out) hist_out[i] = done[i];
        if (s_out) s_out[i] = s[i];
    }
    if (rounds_out) *rounds_out = rounds;
    if (transport_ms_out) *transport_ms_out = transport_ms;
    if (sequences_out) *sequences_out = sequences;
    return GPUMCD_OK;
}

static gpumcd_status simulate_impl(gpumcd_ctx *c, int32_t phantom_id, const gpumcd_source *src, uint64_t n,
                                   uint64_t seed, double target, double *dose, double *sigma, bool host,
                                   cudaStream_t s, gpumcd_run_stats *stats) {
    if (!c || n == 0 || !(target >= 0.0)) return GPUMCD_ERR_INVALID_ARG;
    int32_t pid = 0;
    ST(gpumcd_plan_open(c, phantom_id, src, seed, 32, &pid));
    gpumcd_status st = GPUMCD_OK;
    gpumcd_run_stats rs{};
    const uint64_t cap = target > 0.0 ? std::max<uint64_t>(16 * n, 1000000000ull) : n;
    uint64_t done = 0;
    do {
        st = gpumcd_run(c, 1, &pid, &n, s);
        if (st != GPUMCD_OK) break;
        done += n;
        if (target <= 0.0) break;
        st = gpumcd_plan_result(c, pid, 0.5, nullptr, nullptr, s, &rs);
        if (st != GPUMCD_OK) break;
    } while (rs.s_thr > target && done + n <= cap);
    const uint64_t nvox = c->phantoms.at(phantom_id).nvox;
    if (st == GPUMCD_OK) {
        if (host) {
            st = gpumcd_plan_result(c, pid, 0.5, nullptr, nullptr, s, &rs);
            if (st == GPUMCD_OK) {
                const double *td = (const double *)c->fold_tmp.p;
                cudaError_t e = cudaSuccess;
                if (dose) e = cudaMemcpyAsync(dose, td, nvox * 8, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess && sigma) e = cudaMemcpyAsync(sigma, td + nvox, nvox * 8, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) st = cuda_status(e);
            }
        } else {
            st = gpumcd_plan_result(c, pid, 0.5, dose, sigma, s, &rs);
        }
    }
    if (st == GPUMCD_OK && stats) *stats = rs;
    gpumcd_plan_close(c, pid);
    return st;
}

gpumcd_status gpumcd_simulate(gpumcd_ctx *c, int32_t phantom_id, const gpumcd_source *src, uint64_t n,
                              uint64_t seed, double target, double *dose, double *sigma, gpumcd_run_stats *stats) {
    if (!c) return GPUMCD_ERR_INVALID_ARG;
    return simulate_impl(c, phantom_id, src, n, seed, target, dose, sigma, true, c->stream, stats);
}

gpumcd_status gpumcd_simulate_device(gpumcd_ctx *c, int32_t phantom_id, const gpumcd_source *src, uint64_t n,
                                     uint64_t seed, double target, double *dose, double *sigma, void *stream,
                                     gpumcd_run_stats *stats) {
    if (!c) return GPUMCD_ERR_INVALID_ARG;
    return simulate_impl(c, phantom_id, src, n, seed, target, dose, sigma, false, pick(c, stream), stats);
}

gpumcd_status gpumcd_memory(gpumcd_ctx *c, uint64_t *used, uint64_t *budget) {
    if (!c || !used || !budget) return GPUMCD_ERR_INVALID_ARG;
    *used = c->used;
    *budget = c->budget;
    return GPUMCD_OK;
}

gpumcd_status gpumcd_set_launch(gpumcd_ctx *c, const gpumcd_launch *l) {
    if (!c || !l) return GPUMCD_ERR_INVALID_ARG;
    if (any_busy(c)) return GPUMCD_ERR_STATE;
    gpumcd_launch n = c->launch;
    if (l->block_threads) n.block_threads = l->block_threads;
    if (l->blocks_per_sm) n.blocks_per_sm = l->blocks_per_sm;
    if (l->stack_capacity) n.stack_capacity = l->stack_capacity;
    if (l->switch_high) n.switch_high = l->switch_high;
    if (l->refill_low) n.refill_low = l->refill_low;
    if (l->chunk) n.chunk = l->chunk;
    if (l->overflow_capacity) n.overflow_capacity = l->overflow_capacity;
    n.flags = l->flags;
    if (l->refill_period) n.refill_period = l->refill_period;
    if (n.block_threads % 32 || n.block_threads < 32 || n.block_threads > 1024) return GPUMCD_ERR_INVALID_ARG;
    if (n.blocks_per_sm < 1 || n.blocks_per_sm > 4) return GPUMCD_ERR_INVALID_ARG;
    // every kernel is built for at most 1024 threads per SM (64 registers each)
    if (n.block_threads * n.blocks_per_sm > 1024) return GPUMCD_ERR_INVALID_ARG;
    if (n.stack_capacity < 128 || n.stack_capacity > (1u << 16)) return GPUMCD_ERR_INVALID_ARG;
    if (n.switch_high < 32 || n.switch_high > n.stack_capacity) return GPUMCD_ERR_INVALID_ARG;
    if (n.refill_low > 32 || n.chunk < 1 || n.chunk > 4096) return GPUMCD_ERR_INVALID_ARG;
    if (n.overflow_capacity < 64 || n.overflow_capacity > (1u << 26)) return GPUMCD_ERR_INVALID_ARG;
    // the profiling, warp-aggregating, refill-policy and photon-only kernels
    // are separate instantiations: at most one of them at a time
    const int special = ((n.flags & GPUMCD_LAUNCH_PROFILE) != 0u) + ((n.flags & GPUMCD_LAUNCH_WARP_AGGREGATE) != 0u) +
                        (n.refill_period != 1u) + ((n.flags & GPUMCD_LAUNCH_KERMA) != 0u);
    if (special > 1) return GPUMCD_ERR_INVALID_ARG;
    c->launch = n;
    return GPUMCD_OK;
}

gpumcd_status gpumcd_get_launch(gpumcd_ctx *c, gpumcd_launch *l) {
    if (!c || !l) return GPUMCD_ERR_INVALID_ARG;
    *l = c->launch;
    return GPUMCD_OK;
}

gpumcd_status gpumcd_get_tables(gpumcd_ctx *c, int32_t which, float *out, int32_t *count) {
    if (!c || !count) return GPUMCD_ERR_INVALID_ARG;
    if (!c->tables) return GPUMCD_ERR_STATE;
    int n = 0;
    if (which == 0) n = NMAT * 3 * G;
    else if (which == 1) n = NMAT * 4 * G;
    else if (which == 2) n = G_MS;
    else if (which == 3) n = 2 * G;
    else return GPUMCD_ERR_INVALID_ARG;
    *count = n;
    if (!out) return GPUMCD_OK;
    ST(set_device(c));
    if (which == 3) {
        DevBuf tmp;
        ST(dev_alloc(c, tmp, 2 * G * 4));
        cudaError_t e = launch_grid_energies(c->geom, (float *)tmp.p, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp.p, 2 * G * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        dev_free(c, tmp);
        return cuda_status(e);
    }
    // the device keeps one block per material; the diagnostic layout is per table kind
    std::vector<float> all(TAB_FLOATS);
    CK(cudaMemcpyAsync(all.data(), c->tab.p, TAB_BYTES, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (which == 2) {
        memcpy(out, all.data() + TAB_MS, (size_t)G_MS * 4);
    } else {
        const int k = which == 0 ? 3 : 4;
        for (int m = 0; m < NMAT; ++m)
            memcpy(out + (size_t)m * k * G, all.data() + (which == 0 ? tab_ph(m) : tab_el(m)), (size_t)k * G * 4);
    }
    return GPUMCD_OK;
}

gpumcd_status gpumcd_debug_sample(gpumcd_ctx *c, int32_t kind, double p0, int32_t material,
                                  const gpumcd_source *src, uint64_t n, uint64_t seed, float *out) {
    if (!c || !out || n == 0 || n > (1ull << 28) || kind < 0 || kind > 6) return GPUMCD_ERR_INVALID_ARG;
    if (!c->tables) return GPUMCD_ERR_STATE;
    if (material < 0 || material >= c->n_mat) return GPUMCD_ERR_INVALID_ARG;
    if (kind == 5 && (!valid_source(c, src) || src->n_spectrum < 1)) return GPUMCD_ERR_INVALID_ARG;
    if (kind != 5 && !(p0 > 0.0)) return GPUMCD_ERR_INVALID_ARG;
    if (kind == 2 && !(p0 > 2.0 * c->phys.t_c)) return GPUMCD_ERR_INVALID_ARG;
    if (kind == 3 && !(p0 > c->phys.k_c)) return GPUMCD_ERR_INVALID_ARG;
    ST(set_device(c));
    DevBuf o, spec, tmp;
    gpumcd_status st = dev_alloc(c, o, n * 4);
    cudaError_t e = cudaSuccess;
    int ns = 0;
    if (st == GPUMCD_OK && kind == 5) {
        ns = src->n_spectrum;
        st = dev_alloc(c, spec, (size_t)2 * (ns + 1) * 4);
        if (st == GPUMCD_OK) st = dev_alloc(c, tmp, (size_t)(2 * ns + 1) * 8);
        if (st == GPUMCD_OK) {
            double *d = (double *)tmp.p;
            e = cudaMemcpyAsync(d, src->spectrum_edges, (ns + 1) * 8, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d + ns + 1, src->spectrum_weights, ns * 8, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = launch_spectrum(d, d + ns + 1, ns, (float *)spec.p, c->stream);
        }
    }
    if (st == GPUMCD_OK && e == cudaSuccess)
        e = launch_debug_sample((const float *)c->tab.p, c->dphys, kind, (float)p0, material,
                                (const float *)spec.p, ns, n, seed, (float *)o.p, c->stream);
    if (st == GPUMCD_OK && e == cudaSuccess) e = cudaMemcpyAsync(out, o.p, n * 4, cudaMemcpyDeviceToHost, c->stream);
    if (st == GPUMCD_OK && e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, o);
    dev_free(c, spec);
    dev_free(c, tmp);
    if (st != GPUMCD_OK) return st;
    return cuda_status(e);
}

gpumcd_status gpumcd_debug_counters(gpumcd_ctx *c, uint64_t *out, int32_t *count) {
    if (!c || !count) return GPUMCD_ERR_INVALID_ARG;
    *count = CNT_N;
    if (!out) return GPUMCD_OK;
    if (!c->have_last) return GPUMCD_ERR_STATE;
    for (int i = 0; i < CNT_N; ++i) out[i] = c->last.counters[i];
    return GPUMCD_OK;
}

gpumcd_status gpumcd_debug_majorants(gpumcd_ctx *c, int32_t phantom, float *majorants, float *rho_max) {
    if (!c || !majorants || !rho_max) return GPUMCD_ERR_INVALID_ARG;
    auto it = c->phantoms.find(phantom);
    if (it == c->phantoms.end()) return GPUMCD_ERR_NOT_FOUND;
    ST(set_device(c));
    CK(cudaMemcpyAsync(majorants, it->second.maj.p, MAJ_FLOATS * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(rho_max, it->second.rhomax.p, NMAT * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return GPUMCD_OK;
}

gpumcd_status gpumcd_debug_philox(gpumcd_ctx *c, const uint32_t *ctr, const uint32_t key[2], uint64_t n,
                                  int32_t use_curand, uint32_t *out) {
    if (!c || !ctr || !key || !out || n == 0 || n > (1ull << 24)) return GPUMCD_ERR_INVALID_ARG;
    ST(set_device(c));
    DevBuf dc, dout;
    gpumcd_status st = dev_alloc(c, dc, n * 16);
    if (st == GPUMCD_OK) st = dev_alloc(c, dout, n * 16);
    cudaError_t e = cudaSuccess;
    if (st == GPUMCD_OK) {
        e = cudaMemcpyAsync(dc.p, ctr, n * 16, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = launch_philox((const uint32_t *)dc.p, make_uint2(key[0], key[1]), n, use_curand, (uint32_t *)dout.p,
                              c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout.p, n * 16, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    dev_free(c, dc);
    dev_free(c, dout);
    if (st != GPUMCD_OK) return st;
    return cuda_status(e);
}

}  // extern "C"
