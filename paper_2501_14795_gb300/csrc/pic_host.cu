// Host runtime behind the C ABI of include/pic.h: configuration checks,
// device memory, TMA descriptors, the per-step launch sequence, CUDA-graph
// capture (one graph per buffer parity), timing events and diagnostics.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "host_internal.h"

using namespace pic;

namespace pic {
namespace host {

pic_status fail(pic_sim* s, pic_status code, const char* fmt, ...) {
    if (s) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        s->err = buf;
    }
    return code;
}

#define CK(call) PIC_CK(sim, call)

// Host-side fault injection for the allocation-failure paths: with
// PIC_FAULT=alloc in the environment (read at every call, so it can be set
// around a single call) each device allocation of a simulation reports
// cudaErrorMemoryAllocation without calling cudaMalloc.  Nothing reaches the
// GPU; the clean-up and the PIC_ENOMEM report run as they would.
bool fault_alloc() {
    const char* v = getenv("PIC_FAULT");
    return v && strcmp(v, "alloc") == 0;
}

template <class P>
cudaError_t dalloc(P** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (fault_alloc()) return cudaErrorMemoryAllocation;
    return cudaMalloc((void**)p, sizeof(P) * count);
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3D map over the six E|B components: x = column (P), y = row (R), z = component;
// box = the tile's halo, (T+8) columns x (T+3) rows x 6 components.
bool make_field_map(CUtensorMap* map, const Geom& g, float* base) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)g.P, (cuuint64_t)g.R, 6};
    cuuint64_t strides[2] = {(cuuint64_t)g.P * 4, (cuuint64_t)g.cstride * 4};
    cuuint32_t box[3] = {(cuuint32_t)(g.T + 8), (cuuint32_t)(g.T + 3), 6};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The field kernel's TMA boxes: E or B of F (3 of its 6 components) as
// 40 x 19 x 3 and J as 36 x 17 x 3 (the x extents multiples of 16 bytes).
bool make_yee_maps(CUtensorMap* mapF, CUtensorMap* mapJ, const Geom& g, float* F, float* J) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t strides[2] = {(cuuint64_t)g.P * 4, (cuuint64_t)g.cstride * 4};
    cuuint32_t estr[3] = {1, 1, 1};
    cuuint64_t dF[3] = {(cuuint64_t)g.P, (cuuint64_t)g.R, 6};
    cuuint32_t bF[3] = {40, 19, 3};
    CUresult r = enc(mapF, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, F, dF, strides, bF, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    cuuint64_t dJ[3] = {(cuuint64_t)g.P, (cuuint64_t)g.R, 3};
    cuuint32_t bJ[3] = {36, 17, 3};
    r = enc(mapJ, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, J, dJ, strides, bJ, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Geometry of a configuration (tile size included).
void set_geometry(Geom& g, const pic_config& c) {
    g.nx = c.nx;
    g.ny = c.ny;
    g.T = c.tile;
    g.ntx = c.nx / c.tile;
    g.nty = c.ny / c.tile;
    g.ntiles = g.ntx * g.nty;
    g.P = c.nx + 2 * GX;
    g.R = c.ny + 3;
    g.cstride = (long long)g.P * g.R;
    g.cx = (float)(c.dt / c.dx);
    g.cy = (float)(c.dt / c.dy);
    g.hdt_dx = (float)(0.5 * c.dt / c.dx);
    g.hdt_dy = (float)(0.5 * c.dt / c.dy);
    g.dt_dx = (float)(c.dt / c.dx);
    g.dt_dy = (float)(c.dt / c.dy);
    g.dt = (float)c.dt;
    g.dx = c.dx;
    g.dy = c.dy;
    g.dtd = c.dt;
    g.open_x = 0;
    g.pad_g = 0;
}

// Per-tile bookkeeping of a species (tile bookmarks, leaver counters by
// destination, displaced counts), zeroed.
cudaError_t alloc_tile_arrays(SpeciesDev& s, const Geom& g, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2; ++b) {
        if (e == cudaSuccess) e = dalloc(&s.off[b], g.ntiles + 1);
        if (e == cudaSuccess) e = dalloc(&s.leave[b], g.ntiles);
        if (e == cudaSuccess) e = dalloc(&s.dirc[b], 8 * (size_t)g.ntiles);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(s.off[b], 0, sizeof(int32_t) * (g.ntiles + 1), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(s.leave[b], 0, sizeof(int32_t) * g.ntiles, st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(s.dirc[b], 0, sizeof(int32_t) * 8 * g.ntiles, st);
    }
    if (e == cudaSuccess) e = dalloc(&s.evict, g.ntiles);
    if (e == cudaSuccess) e = dalloc(&s.ldir, 9 * (size_t)g.ntiles);
    return e;
}

void free_tile_arrays(SpeciesDev& s) {
    for (int b = 0; b < 2; ++b) {
        dfree(s.off[b]);
        dfree(s.leave[b]);
        dfree(s.dirc[b]);
        s.off[b] = s.leave[b] = s.dirc[b] = nullptr;
    }
    dfree(s.evict);
    dfree(s.ldir);
    s.evict = s.ldir = nullptr;
}

void free_species(SpeciesDev& s) {
    void* ptrs[] = {s.cell, s.x,   s.y,   s.ux,  s.uy,  s.uz,   s.id,    s.ocell, s.ox, s.oy,
                    s.oux,  s.ouy, s.ouz, s.oid, s.hole, s.fslot, s.isrc, s.odir,  s.lsort};
    for (void* p : ptrs) dfree(p);
    s.cell = s.id = s.ocell = s.oid = s.hole = s.fslot = s.isrc = s.lsort = nullptr;
    s.odir = nullptr;
    s.x = s.y = s.ux = s.uy = s.uz = s.ox = s.oy = s.oux = s.ouy = s.ouz = nullptr;
    s.cap = 0;
}

// The particle kernels copy batches of up to 1024 particles from the 16-byte
// aligned index at or below the batch start, so every array carries this many
// spare elements past its capacity.
constexpr int64_t kParticlePad = 1024 + 64;

cudaError_t alloc_particles(SpeciesDev& s, int64_t cap) {
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p) {
        if (e == cudaSuccess) e = dalloc(p, (size_t)(cap + kParticlePad));
    };
    A(&s.cell); A(&s.x); A(&s.y); A(&s.ux); A(&s.uy); A(&s.uz); A(&s.id);
    A(&s.ocell); A(&s.ox); A(&s.oy); A(&s.oux); A(&s.ouy); A(&s.ouz); A(&s.oid);
    A(&s.hole); A(&s.fslot); A(&s.isrc); A(&s.odir); A(&s.lsort);
    if (e == cudaSuccess) s.cap = cap;
    return e;
}

void invalidate_graphs(pic_sim* sim) {
    for (int b = 0; b < 2; ++b) {
        if (sim->gexec[b]) cudaGraphExecDestroy(sim->gexec[b]);
        if (sim->graph[b]) cudaGraphDestroy(sim->graph[b]);
        sim->gexec[b] = nullptr;
        sim->graph[b] = nullptr;
        for (auto& nd : sim->ev_node[b]) nd = nullptr;
    }
    sim->gen += 1;
}

// CTAs per tile in the particle advance: tiles holding many particles are
// split so that every CTA takes about kChunkParticles (the grid then has many
// CTAs per SM and the hardware balances them); one CTA per tile otherwise.
constexpr int kMaxChunks = 1024;

// With the fixed-point J tiles a CTA item holds at most kMaxItemBatches
// batches of blockDim particles: the tiles' scale is set by the particles an
// item can deposit, so this bounds the quantum at 2^-18 |qtilde|.
constexpr int kMaxItemBatches = 64;

int chunks_per_tile(const pic_sim* sim) {
    int64_t nmax = 0;
    for (int k = 0; k < sim->cfg.n_species; ++k) nmax = std::max(nmax, sim->sp[k].n);
    const int64_t per_tile = sim->g.ntiles ? nmax / sim->g.ntiles : 0;
    int64_t chunk = sim->cfg.chunk;
    if (!(sim->cfg.flags & PIC_FP32_J))
        chunk = std::min<int64_t>(chunk, (int64_t)kMaxItemBatches * sim->cfg.threads);
    const int64_t c = (per_tile + chunk - 1) / chunk;
    return (int)std::min<int64_t>(std::max<int64_t>(c, 1), kMaxChunks);
}

PushParams push_params(const pic_sim* sim, int b) {
    PushParams p;
    memset(&p, 0, sizeof p);
    p.g = sim->g;
    p.J = sim->J[b];
    p.nsp = sim->cfg.n_species;
    p.track_ids = (sim->cfg.flags & PIC_TRACK_IDS) ? 1 : 0;
    p.fp32_j = (sim->cfg.flags & PIC_FP32_J) ? 1 : 0;
    for (int k = 0; k < p.nsp; ++k) {
        const SpeciesDev& s = sim->sp[k];
        PushSpecies& q = p.sp[k];
        q.off = s.off[b];
        q.cell = s.cell; q.id = s.id; q.ocell = s.ocell; q.oid = s.oid; q.hole = s.hole;
        q.leave = s.leave[b]; q.dirc = s.dirc[b]; q.odir = s.odir;
        q.x = s.x; q.y = s.y; q.ux = s.ux; q.uy = s.uy; q.uz = s.uz;
        q.ox = s.ox; q.oy = s.oy; q.oux = s.oux; q.ouy = s.ouy; q.ouz = s.ouz;
        q.tem = s.tem; q.qjx = s.qjx; q.qjy = s.qjy; q.qjz = s.qjz; q.ke_w = s.ke_w;
    }
    p.chunks = chunks_per_tile(sim);
    p.hist_k = sim->hist_k;
    p.st = sim->st;
    return p;
}

SortParams sort_params(const pic_sim* sim, int b) {
    SortParams p;
    memset(&p, 0, sizeof p);
    p.g = sim->g;
    p.nsp = sim->cfg.n_species;
    p.track_ids = (sim->cfg.flags & PIC_TRACK_IDS) ? 1 : 0;
    for (int k = 0; k < p.nsp; ++k) {
        const SpeciesDev& s = sim->sp[k];
        SortSpecies& q = p.sp[k];
        q.off_old = s.off[b];
        q.off_new = s.off[1 - b];
        q.cell = s.cell; q.id = s.id; q.ocell = s.ocell; q.oid = s.oid; q.hole = s.hole;
        q.fslot = s.fslot; q.isrc = s.isrc; q.leave = s.leave[b]; q.dirc = s.dirc[b];
        q.leave_next = s.leave[1 - b]; q.dirc_next = s.dirc[1 - b]; q.evict = s.evict;
        q.odir = s.odir; q.lsort = s.lsort; q.ldir = s.ldir;
        q.x = s.x; q.y = s.y; q.ux = s.ux; q.uy = s.uy; q.uz = s.uz;
        q.ox = s.ox; q.oy = s.oy; q.oux = s.oux; q.ouy = s.ouy; q.ouz = s.ouz;
        q.n = (int)s.n;
        q.cap = (int)std::min<int64_t>(s.cap, 0x7fffffff);
        q.inj_k = s.inj_k;
        q.inj_u[0] = s.inj_u[0];
        q.inj_u[1] = s.inj_u[1];
        q.inj_u[2] = s.inj_u[2];
        q.inj_x0 = s.inj_x0;
    }
    p.hist_e = sim->hist_e;
    p.hist_b = sim->hist_b;
    p.hist_k = sim->hist_k;
    p.st = sim->st;
    return p;
}

YeeParams yee_params(const pic_sim* sim, int b, int chunks) {
    YeeParams yp;
    memset(&yp, 0, sizeof yp);
    yp.g = sim->g;
    yp.Fin = sim->F[b];
    yp.Fout = sim->F[1 - b];
    yp.J = sim->J[b];
    yp.Jnext = sim->J[1 - b];
    yp.hist_e = sim->hist_e;
    yp.hist_b = sim->hist_b;
    yp.st = sim->st;
    yp.zero_all = chunks > 1;
    return yp;
}

// Enqueue one step at parity b.  Returns the number of kernels launched or
// -1 on a launch error (message in sim->err).  ev, when non-null, holds the
// kStepEvents events recorded before the particle advance, after it, after
// the re-sort and after the field advance (external event records inside a
// capture).
int enqueue_step(pic_sim* sim, cudaStream_t s, int b, const cudaEvent_t* ev, bool capturing) {
    const int threads = sim->cfg.threads;
    const PushParams pp = push_params(sim, b);
    const SortParams sp = sort_params(sim, b);
    const YeeParams yp = yee_params(sim, b, pp.chunks);
    int n = 0;
    cudaError_t e;
    const unsigned rec = capturing ? cudaEventRecordExternal : 0u;
    if (ev && (e = cudaEventRecordWithFlags(ev[0], s, rec)) != cudaSuccess) goto bad;
    e = (sim->cfg.flags & PIC_STRICT_FP) ? launch_push_strict(&sim->fmap[b], pp, threads, s)
                                         : launch_push_fast(&sim->fmap[b], pp, threads, s);
    if (e != cudaSuccess) goto bad;
    n += sim->g.ntiles > 0;
    if (ev && (e = cudaEventRecordWithFlags(ev[1], s, rec)) != cudaSuccess) goto bad;
    if ((e = launch_scan(sp, s)) != cudaSuccess) goto bad;
    n += (sp.nsp > 0 && sim->g.ntiles > 0) ? 2 : 1;  // count + scan
    // Fork.  The field branch needs the deposit and the scan (it adds its
    // energies into the history slot of the level the scan moved to) but not
    // the particles' places, and the eviction and fill touch no field: the
    // field advance runs beside them, and the next step starts after both.
    if ((e = cudaEventRecord(sim->ev_fork, s)) != cudaSuccess) goto bad;
    if ((e = cudaStreamWaitEvent(sim->side_stream, sim->ev_fork, 0)) != cudaSuccess) goto bad;
    if ((e = launch_evict(sp, threads, s)) != cudaSuccess) goto bad;
    if ((e = launch_fill(sp, threads, s)) != cudaSuccess) goto bad;
    n += (sp.nsp > 0 && sim->g.ntiles > 0) ? 2 : 0;
    if (ev && (e = cudaEventRecordWithFlags(ev[2], s, rec)) != cudaSuccess) goto bad;
    if (sim->jfilter) {
        // the current-filter slot of Listing 3.1: after the deposit and its
        // guard-cell reduction, before the field advance
        const int k = sim->jfilter(sim->jfilter_ctx, sim, sim->side_stream, b);
        if (k < 0) return -1;
        n += k;
    }
    if ((e = launch_yee(yp, &sim->ymapF[b], &sim->ymapJ[b], sim->side_stream)) != cudaSuccess)
        goto bad;
    n += 1;
    // join
    if ((e = cudaEventRecord(sim->ev_join, sim->side_stream)) != cudaSuccess) goto bad;
    if ((e = cudaStreamWaitEvent(s, sim->ev_join, 0)) != cudaSuccess) goto bad;
    if (ev && (e = cudaEventRecordWithFlags(ev[3], s, rec)) != cudaSuccess) goto bad;
    return n;
bad:
    sim->err = std::string("kernel launch failed: ") + cudaGetErrorString(e);
    return -1;
}

pic_status build_graph(pic_sim* sim, int b) {
    cudaGraph_t graph = nullptr;
    const bool timing = (sim->cfg.flags & PIC_TIMING) != 0;
    // capture on the private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is launched on the caller's
    CK(cudaStreamBeginCapture(sim->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int n =
        enqueue_step(sim, sim->cap_stream, b, timing ? sim->ev_placeholder : nullptr, true);
    cudaError_t e = cudaStreamEndCapture(sim->cap_stream, &graph);
    if (n < 0) {
        if (graph) cudaGraphDestroy(graph);
        return PIC_ECUDA;
    }
    CK(e);
    sim->launches_per_step = n;
    if (timing) {
        size_t count = 0;
        CK(cudaGraphGetNodes(graph, nullptr, &count));
        std::vector<cudaGraphNode_t> nodes(count);
        CK(cudaGraphGetNodes(graph, nodes.data(), &count));
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            CK(cudaGraphNodeGetType(nd, &ty));
            if (ty != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev;
            CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
            for (int k = 0; k < pic_sim::kStepEvents; ++k)
                if (ev == sim->ev_placeholder[k]) sim->ev_node[b][k] = nd;
        }
    }
    e = cudaGraphInstantiate(&sim->gexec[b], graph, 0);
    sim->graph[b] = graph;
    CK(e);
    return PIC_OK;
}

// The next step's kStepEvents timing events from the pool (grown on demand).
pic_status timing_events(pic_sim* sim, cudaEvent_t** out) {
    constexpr size_t K = pic_sim::kStepEvents;
    const size_t need = K * (sim->ev_used + 1);
    while (sim->ev_pool.size() < need) {
        cudaEvent_t ev;
        CK(cudaEventCreate(&ev));
        sim->ev_pool.push_back(ev);
    }
    *out = sim->ev_pool.data() + K * sim->ev_used;
    sim->ev_used += 1;
    return PIC_OK;
}

pic_status read_state(pic_sim* sim, DevState* h) {
    CK(cudaMemcpyAsync(h, sim->st, sizeof(DevState), cudaMemcpyDeviceToHost, sim->stream));
    CK(cudaStreamSynchronize(sim->stream));
    return PIC_OK;
}

pic_status status_from_bits(pic_sim* sim, unsigned bits) {
    if (bits & ST_TIMEOUT) return fail(sim, PIC_ETIMEOUT, "a bounded device wait ran out");
    if (bits & ST_SORT)
        return fail(sim, PIC_EOVERFLOW, "tile re-sort bookkeeping inconsistent");
    if (bits & ST_PARTICLE)
        return fail(sim, PIC_EPARTICLE,
                    "a particle moved one cell or more in a step or has a non-finite momentum");
    return PIC_OK;
}

pic_status sync_status(pic_sim* sim) {
    DevState h;
    pic_status r = read_state(sim, &h);
    if (r != PIC_OK) return r;
    return status_from_bits(sim, h.status);
}

pic_status refresh_counts(pic_sim* sim) {
    if (!sim->window) return PIC_OK;
    DevState h;
    pic_status r = read_state(sim, &h);
    if (r != PIC_OK) return r;
    for (int k = 0; k < sim->cfg.n_species; ++k) sim->sp[k].n = h.np[k];
    return PIC_OK;
}

// zero the history slots of the current level and record the field energy
pic_status refresh_level_energy(pic_sim* sim) {
    CK(launch_hist_prime(sim->hist_e, sim->hist_b, sim->hist_k, sim->st, sim->stream));
    const long long n = sim->step & (HIST - 1);
    CK(launch_field_energy(sim->g, sim->F[sim->cur], sim->hist_e + n, sim->hist_b + n,
                           sim->stream));
    return PIC_OK;
}

const void* stage_in(pic_sim* sim, const void* src, size_t bytes, void* staging, int on_device,
                     pic_status* st) {
    *st = PIC_OK;
    if (on_device || bytes == 0) return src;
    cudaError_t e = cudaMemcpyAsync(staging, src, bytes, cudaMemcpyHostToDevice, sim->stream);
    if (e != cudaSuccess) {
        *st = fail(sim, PIC_ECUDA, "host-to-device copy failed: %s", cudaGetErrorString(e));
        return nullptr;
    }
    return staging;
}


// the binomial filter in the current-filter slot
int binomial_hook(void*, pic_sim* sim, cudaStream_t s, int b) {
    for (int k = 0; k < sim->binomial_passes; ++k) {
        cudaError_t e = launch_binomial(sim->g, sim->J[b], sim->gtmp, s);
        if (e != cudaSuccess) {
            sim->err = std::string("binomial filter launch failed: ") + cudaGetErrorString(e);
            return -1;
        }
    }
    return 2 * sim->binomial_passes;
}

pic_status retile(pic_sim* sim, int tile) {
    const pic_config& c = sim->cfg;
    if (!(tile == 8 || tile == 16 || tile == 32) || c.nx % tile || c.ny % tile)
        return fail(sim, PIC_EINVAL, "tile %d does not divide the %dx%d grid", tile, c.nx, c.ny);
    if (tile == sim->g.T) return PIC_OK;
    cudaStream_t s = sim->stream;
    {
        pic_status r = refresh_counts(sim);
        if (r != PIC_OK) return r;
    }
    {
        DevState h;
        pic_status r = read_state(sim, &h);
        if (r != PIC_OK) return r;
        if (h.status) return status_from_bits(sim, h.status);
    }
    const bool track = (c.flags & PIC_TRACK_IDS) != 0;
    // stage every species in its out arrays, as the load path expects them
    for (int k = 0; k < c.n_species; ++k) {
        SpeciesDev& S = sim->sp[k];
        if (S.n == 0) continue;
        const size_t b4 = 4 * (size_t)S.n;
        CK(launch_unpack_cells(S.cell, S.n, S.ocell, S.hole, s));
        CK(cudaMemcpyAsync(S.ox, S.x, b4, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(S.oy, S.y, b4, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(S.oux, S.ux, b4, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(S.ouy, S.uy, b4, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(S.ouz, S.uz, b4, cudaMemcpyDeviceToDevice, s));
        if (track) CK(cudaMemcpyAsync(S.isrc, S.id, b4, cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaStreamSynchronize(s));
    invalidate_graphs(sim);
    sim->cfg.tile = tile;
    set_geometry(sim->g, sim->cfg);
    sim->g.open_x = sim->window;
    for (int k = 0; k < c.n_species; ++k) {
        free_tile_arrays(sim->sp[k]);
        CK(alloc_tile_arrays(sim->sp[k], sim->g, s));
    }
    for (int b = 0; b < 2; ++b)
        if (!make_field_map(&sim->fmap[b], sim->g, sim->F[b]))
            return fail(sim, PIC_ECUDA, "cannot encode the field tensor map");
    // the next step deposits into J[cur] with plain stores on the tiles'
    // interiors: it must be all zero for the new tiling
    CK(cudaMemsetAsync(sim->J[sim->cur], 0, 3 * (size_t)sim->g.cstride * 4, s));
    CK(cudaMemsetAsync(&sim->st->load_bad, 0, sizeof(int), s));
    DevState h;
    for (int k = 0; k < c.n_species; ++k) {
        SpeciesDev& S = sim->sp[k];
        CK(launch_load(sim->g, S, track, S.n, S.off[sim->cur], sim->st, s, 0, nullptr, nullptr));
        // the scatter trusts the validated cells: check before it runs
        pic_status r = read_state(sim, &h);
        if (r != PIC_OK) return r;
        if (h.load_bad)
            return fail(sim, PIC_EOVERFLOW, "re-tiling found %d invalid particles", h.load_bad);
        CK(launch_load(sim->g, S, track, S.n, S.off[sim->cur], sim->st, s, 1,
                       track ? S.isrc : nullptr, reinterpret_cast<int32_t*>(sim->rho)));
    }
    pic_status r = read_state(sim, &h);
    if (r != PIC_OK) return r;
    sim->rho_prev_step = -1;
    return status_from_bits(sim, h.status);
}

}  // namespace host
}  // namespace pic

using namespace pic::host;

extern "C" {

pic_status pic_init(const pic_config* cfg, void* cuda_stream, pic_sim** out) {
    if (!out) return PIC_EINVAL;
    *out = nullptr;
    if (!cfg) return PIC_EINVAL;
    pic_config c = *cfg;
    if (c.tile == 0) c.tile = 16;
    if (c.threads == 0) c.threads = 256;
    if (c.chunk == 0) c.chunk = 8192;  // measured on GB300: 4 % faster than 4096 on the Weibel 512^2 case
    if (c.chunk < 16 || c.chunk > (1 << 20)) return PIC_EINVAL;
    if (!(c.tile == 8 || c.tile == 16 || c.tile == 32)) return PIC_EINVAL;
    if (c.threads < 64 || c.threads > 512 || c.threads % 32) return PIC_EINVAL;
    if (c.nx < 8 || c.ny < 8 || c.nx > 32768 || c.ny > 32768) return PIC_EINVAL;
    if (c.nx % c.tile || c.ny % c.tile) return PIC_EINVAL;
    if (c.n_species < 1 || c.n_species > PIC_MAX_SPECIES) return PIC_EINVAL;
    if (!(c.dx > 0 && c.dy > 0 && c.dt > 0) || !std::isfinite(c.dx) || !std::isfinite(c.dy) ||
        !std::isfinite(c.dt))
        return PIC_EINVAL;
    for (int k = 0; k < c.n_species; ++k)
        if (!(c.species[k].density > 0) || !(c.species[k].ppc > 0) ||
            !(c.species[k].q_over_m != 0) || !std::isfinite(c.species[k].q_over_m))
            return PIC_EINVAL;
    // Courant condition, Eq. 1 (c = 1)
    const double lim = 1.0 / std::sqrt(1.0 / (c.dx * c.dx) + 1.0 / (c.dy * c.dy));
    if (!(c.dt < lim)) return PIC_ECFL;

    pic_sim* sim = new pic_sim();
    sim->cfg = c;
    sim->stream = (cudaStream_t)cuda_stream;
    Geom& g = sim->g;
    set_geometry(g, c);

    auto cleanup_fail = [&](pic_status code, const char* what, cudaError_t e) {
        pic_destroy(sim);
        (void)what;
        (void)e;
        return code;
    };
    cudaError_t e = cudaSuccess;
    const size_t gsz = (size_t)g.cstride;
    for (int b = 0; b < 2; ++b) {
        if (e == cudaSuccess) e = dalloc(&sim->F[b], 6 * gsz);
        if (e == cudaSuccess) e = dalloc(&sim->J[b], 3 * gsz);
        if (e == cudaSuccess) e = cudaMemsetAsync(sim->F[b], 0, 6 * gsz * 4, sim->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(sim->J[b], 0, 3 * gsz * 4, sim->stream);
    }
    const size_t ncell = (size_t)c.nx * c.ny;
    if (e == cudaSuccess) e = dalloc(&sim->gtmp, 3 * ncell);
    if (e == cudaSuccess) e = dalloc(&sim->rho, ncell);
    if (e == cudaSuccess) e = dalloc(&sim->rho_prev, ncell);
    if (e == cudaSuccess) e = dalloc(&sim->hist_e, HIST);
    if (e == cudaSuccess) e = dalloc(&sim->hist_b, HIST);
    if (e == cudaSuccess) e = dalloc(&sim->hist_k, HIST);
    if (e == cudaSuccess) e = dalloc(&sim->dred, 8);
    if (e == cudaSuccess) e = dalloc(&sim->st, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(sim->st, 0, sizeof(DevState), sim->stream);
    // NaN everywhere: levels never recorded read as NaN
    if (e == cudaSuccess) e = cudaMemsetAsync(sim->hist_e, 0xff, HIST * 8, sim->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sim->hist_b, 0xff, HIST * 8, sim->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sim->hist_k, 0xff, HIST * 8, sim->stream);
    for (int k = 0; k < c.n_species && e == cudaSuccess; ++k) {
        SpeciesDev& s = sim->sp[k];
        memset(&s, 0, sizeof s);
        if (e == cudaSuccess) e = alloc_tile_arrays(s, g, sim->stream);
        if (e == cudaSuccess) e = dalloc(&s.cursor, (size_t)c.nx * c.ny);
        const auto& sc = c.species[k];
        const double qt = (sc.q_over_m > 0 ? 1.0 : -1.0) * sc.density / sc.ppc;
        s.qtilde = qt;
        s.tem = (float)(0.5 * sc.q_over_m * c.dt);
        s.qjx = (float)(qt * c.dx / c.dt);
        s.qjy = (float)(qt * c.dy / c.dt);
        s.qjz = (float)qt;
        s.ke_w = qt / sc.q_over_m * c.dx * c.dy;
    }
    if (e != cudaSuccess) return cleanup_fail(e == cudaErrorMemoryAllocation ? PIC_ENOMEM : PIC_ECUDA,
                                              "alloc", e);
    for (int b = 0; b < 2; ++b)
        if (!make_field_map(&sim->fmap[b], g, sim->F[b]) ||
            !make_yee_maps(&sim->ymapF[b], &sim->ymapJ[b], g, sim->F[b], sim->J[b]))
            return cleanup_fail(PIC_ECUDA, "tmap", e);
    {
        // raise the particle kernels' shared-memory limit before any capture
        PushParams p0;
        memset(&p0, 0, sizeof p0);
        p0.g = g;
        if (launch_push_fast(nullptr, p0, c.threads, sim->stream) != cudaSuccess ||
            launch_push_strict(nullptr, p0, c.threads, sim->stream) != cudaSuccess ||
            init_grid_kernels() != cudaSuccess)
            return cleanup_fail(PIC_ECUDA, "smem attribute", e);
    }
    if (cudaStreamCreateWithFlags(&sim->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sim->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sim->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sim->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return cleanup_fail(PIC_ECUDA, "stream", e);
    if (c.flags & PIC_TIMING)
        for (int k = 0; k < pic_sim::kStepEvents; ++k)
            if (cudaEventCreate(&sim->ev_placeholder[k]) != cudaSuccess)
                return cleanup_fail(PIC_ECUDA, "event", e);
    if (refresh_level_energy(sim) != PIC_OK) return cleanup_fail(PIC_ECUDA, "energy", e);
    if (cudaStreamSynchronize(sim->stream) != cudaSuccess)
        return cleanup_fail(PIC_ECUDA, "sync", e);
    *out = sim;
    return PIC_OK;
}

pic_status pic_load_particles(pic_sim* sim, int species, int64_t n, const int32_t* ix,
                              const int32_t* iy, const float* x, const float* y,
                              const float* ux, const float* uy, const float* uz,
                              const int32_t* id, int on_device) {
    if (!sim) return PIC_EINVAL;
    sim->err.clear();
    if (species < 0 || species >= sim->cfg.n_species)
        return fail(sim, PIC_EINVAL, "species %d out of range", species);
    if (n < 0 || n > 0x7fffffffLL) return fail(sim, PIC_EINVAL, "bad particle count %lld", (long long)n);
    if (n > 0 && (!ix || !iy || !x || !y || !ux || !uy || !uz))
        return fail(sim, PIC_EINVAL, "null particle array");
    cudaStream_t s = sim->stream;
    SpeciesDev& S = sim->sp[species];
    const bool track = (sim->cfg.flags & PIC_TRACK_IDS) != 0;
    // stage into the out arrays of a (possibly new) allocation
    SpeciesDev W = S;
    const int64_t need = sim->window ? std::max<int64_t>(n, S.want_cap) : n;
    if (need > 0x7fffffffLL)
        return fail(sim, PIC_EINVAL, "capacity %lld above 2^31-1", (long long)need);
    const bool grow = need > S.cap;
    if (grow) {
        SpeciesDev fresh = S;
        fresh.cell = fresh.id = fresh.ocell = fresh.oid = fresh.hole = fresh.fslot = fresh.isrc =
            fresh.lsort = nullptr;
        fresh.odir = nullptr;
        fresh.x = fresh.y = fresh.ux = fresh.uy = fresh.uz = nullptr;
        fresh.ox = fresh.oy = fresh.oux = fresh.ouy = fresh.ouz = nullptr;
        fresh.cap = 0;
        cudaError_t e = alloc_particles(fresh, need);
        if (e != cudaSuccess) {
            free_species(fresh);
            return fail(sim, PIC_ENOMEM, "cannot allocate %lld particles", (long long)need);
        }
        W = fresh;
    }
    const size_t b4 = 4 * (size_t)n;
    auto copy_in = [&](void* dst, const void* src) -> cudaError_t {
        if (n == 0) return cudaSuccess;
        return cudaMemcpyAsync(dst, src, b4, on_device ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice, s);
    };
    cudaError_t e = cudaSuccess;
    // staging: ix -> ocell, iy -> hole, x.. -> ox.., ids -> isrc
    if (e == cudaSuccess) e = copy_in(W.ocell, ix);
    if (e == cudaSuccess) e = copy_in(W.hole, iy);
    if (e == cudaSuccess) e = copy_in(W.ox, x);
    if (e == cudaSuccess) e = copy_in(W.oy, y);
    if (e == cudaSuccess) e = copy_in(W.oux, ux);
    if (e == cudaSuccess) e = copy_in(W.ouy, uy);
    if (e == cudaSuccess) e = copy_in(W.ouz, uz);
    if (e == cudaSuccess && track && id) e = copy_in(W.isrc, id);
    if (e == cudaSuccess) e = cudaMemsetAsync(&sim->st->load_bad, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_load(sim->g, W, track, n, W.off[sim->cur], sim->st, s, 0, nullptr, nullptr);
    DevState h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sim->st, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess || h.load_bad) {
        if (grow) free_species(W);
        if (e != cudaSuccess)
            return fail(sim, PIC_ECUDA, "particle load failed: %s", cudaGetErrorString(e));
        return fail(sim, PIC_EINVAL, "%d particles with a cell outside the grid, an offset outside [0,1) or a non-finite momentum",
                    h.load_bad);
    }
    // the FP64 charge-density buffer (2 nx*ny ints, nx*ny >= 64) serves as the
    // cell-offset scratch (nx*ny + 2 + 2 ceil(nx*ny / 4096) ints)
    e = launch_load(sim->g, W, track, n, W.off[sim->cur], sim->st, s, 1,
                    (track && id) ? W.isrc : nullptr, reinterpret_cast<int32_t*>(sim->rho));
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        if (grow) free_species(W);
        return fail(sim, PIC_ECUDA, "particle scatter failed: %s", cudaGetErrorString(e));
    }
    if (grow) {
        SpeciesDev old = S;
        free_species(old);
    }
    W.n = n;
    S = W;
    // leaver counters of the next step's parity start from zero (a restore
    // may put the simulation back on a parity whose counters were in use)
    CK(cudaMemsetAsync(S.leave[sim->cur], 0, sizeof(int32_t) * sim->g.ntiles, s));
    CK(cudaMemsetAsync(S.dirc[sim->cur], 0, sizeof(int32_t) * 8 * sim->g.ntiles, s));
    {
        const long long np = n;  // the device count (it changes with the moving window)
        CK(cudaMemcpyAsync(&sim->st->np[species], &np, sizeof np, cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(&sim->st->removed[species], 0, sizeof(long long), s));
        CK(cudaStreamSynchronize(s));
    }
    invalidate_graphs(sim);
    sim->rho_prev_step = -1;
    pic_status r = refresh_level_energy(sim);
    if (r != PIC_OK) return r;
    CK(cudaStreamSynchronize(s));
    return PIC_OK;
}

pic_status pic_set_fields(pic_sim* sim, const float* E, const float* B, int on_device) {
    if (!sim) return PIC_EINVAL;
    sim->err.clear();
    const size_t bytes = 3 * (size_t)sim->g.nx * sim->g.ny * 4;
    const float* srcs[2] = {E, B};
    for (int f = 0; f < 2; ++f) {
        if (!srcs[f]) continue;
        pic_status st;
        const float* src = (const float*)stage_in(sim, srcs[f], bytes, sim->gtmp, on_device, &st);
        if (st != PIC_OK) return st;
        CK(launch_set_grid(sim->g, sim->F[sim->cur] + 3 * f * sim->g.cstride, 3, src,
                           sim->stream));
        CK(cudaStreamSynchronize(sim->stream));
    }
    if (sim->window) CK(launch_zero_x_guards(sim->g, sim->F[sim->cur], 6, sim->stream));
    sim->rho_prev_step = -1;
    pic_status r = refresh_level_energy(sim);
    if (r != PIC_OK) return r;
    CK(cudaStreamSynchronize(sim->stream));
    return PIC_OK;
}

pic_status pic_step(pic_sim* sim, int nsteps) {
    if (!sim) return PIC_EINVAL;
    if (nsteps < 0) return fail(sim, PIC_EINVAL, "negative step count");
    sim->err.clear();
    const bool timing = (sim->cfg.flags & PIC_TIMING) != 0;
    const bool graph = (sim->cfg.flags & PIC_NO_GRAPH) == 0;
    for (int k = 0; k < nsteps; ++k) {
        const int b = sim->cur;
        cudaEvent_t* ev = nullptr;
        if (timing) {
            pic_status r = timing_events(sim, &ev);
            if (r != PIC_OK) return r;
        }
        if (graph) {
            if (!sim->gexec[b]) {
                pic_status r = build_graph(sim, b);
                if (r != PIC_OK) return r;
            }
            if (timing)
                for (int k = 0; k < pic_sim::kStepEvents; ++k)
                    CK(cudaGraphExecEventRecordNodeSetEvent(sim->gexec[b], sim->ev_node[b][k],
                                                            ev[k]));
            CK(cudaGraphLaunch(sim->gexec[b], sim->stream));
            sim->launches += sim->launches_per_step;
        } else {
            const int n = enqueue_step(sim, sim->stream, b, ev, false);
            if (n < 0) return PIC_ECUDA;
            sim->launches += n;
        }
        sim->cur = 1 - b;
        sim->step += 1;
    }
    return PIC_OK;
}

pic_status pic_set_binomial_filter(pic_sim* sim, int passes) {
    if (!sim) return PIC_EINVAL;
    sim->err.clear();
    if (passes < 0 || passes > 64) return fail(sim, PIC_EINVAL, "passes %d not in 0..64", passes);
    if (passes && sim->window)
        return fail(sim, PIC_EINVAL, "the binomial filter is periodic: not with the moving window");
    CK(cudaStreamSynchronize(sim->stream));
    sim->binomial_passes = passes;
    sim->jfilter = passes ? binomial_hook : nullptr;
    sim->jfilter_ctx = nullptr;
    invalidate_graphs(sim);
    return PIC_OK;
}

pic_status pic_get_fields(pic_sim* sim, int which, float* out, int on_device) {
    if (!sim || !out) return PIC_EINVAL;
    sim->err.clear();
    const Geom& g = sim->g;
    const size_t ncell = (size_t)g.nx * g.ny;
    float* dst = on_device ? out : sim->gtmp;
    if (which == 0 || which == 1) {
        CK(launch_get_grid(g, sim->F[sim->cur] + 3 * which * g.cstride, 3, dst, sim->stream));
    } else if (which == 2) {
        CK(launch_get_grid(g, sim->J[1 - sim->cur], 3, dst, sim->stream));
    } else if (which == 3) {
        CK(cudaMemsetAsync(sim->rho, 0, ncell * 8, sim->stream));
        const int32_t* offs[MAX_SPECIES];
        for (int k = 0; k < sim->cfg.n_species; ++k) offs[k] = sim->sp[k].off[sim->cur];
        CK(launch_rho(g, sim->sp, sim->cfg.n_species, offs, sim->rho, sim->stream));
        std::vector<double> h(ncell);
        CK(cudaMemcpyAsync(h.data(), sim->rho, ncell * 8, cudaMemcpyDeviceToHost, sim->stream));
        CK(cudaStreamSynchronize(sim->stream));
        std::vector<float> f(ncell);
        for (size_t k = 0; k < ncell; ++k) f[k] = (float)(h[k] + sim->cfg.background);
        CK(cudaMemcpy(out, f.data(), ncell * 4,
                      on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
        return sync_status(sim);
    } else {
        return fail(sim, PIC_EINVAL, "unknown field %d", which);
    }
    if (!on_device)
        CK(cudaMemcpyAsync(out, sim->gtmp, 3 * ncell * 4, cudaMemcpyDeviceToHost, sim->stream));
    return sync_status(sim);
}

pic_status pic_get_particles(pic_sim* sim, int species, int32_t* ix, int32_t* iy, float* x,
                             float* y, float* ux, float* uy, float* uz, int32_t* id,
                             int64_t* tile_offset, int on_device) {
    if (!sim) return PIC_EINVAL;
    sim->err.clear();
    if (species < 0 || species >= sim->cfg.n_species)
        return fail(sim, PIC_EINVAL, "species %d out of range", species);
    {
        pic_status r = refresh_counts(sim);
        if (r != PIC_OK) return r;
    }
    SpeciesDev& S = sim->sp[species];
    cudaStream_t s = sim->stream;
    const size_t b4 = 4 * (size_t)S.n;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (S.n > 0) {
        // unpack cells into caller buffers (device) or into scratch then copy
        int32_t* dix = on_device ? ix : (ix ? S.ocell : nullptr);
        int32_t* diy = on_device ? iy : (iy ? S.hole : nullptr);
        if (dix || diy) CK(launch_unpack_cells(S.cell, S.n, dix, diy, s));
        if (!on_device && ix) CK(cudaMemcpyAsync(ix, S.ocell, b4, k, s));
        if (!on_device && iy) CK(cudaMemcpyAsync(iy, S.hole, b4, k, s));
        if (x) CK(cudaMemcpyAsync(x, S.x, b4, k, s));
        if (y) CK(cudaMemcpyAsync(y, S.y, b4, k, s));
        if (ux) CK(cudaMemcpyAsync(ux, S.ux, b4, k, s));
        if (uy) CK(cudaMemcpyAsync(uy, S.uy, b4, k, s));
        if (uz) CK(cudaMemcpyAsync(uz, S.uz, b4, k, s));
        if (id && (sim->cfg.flags & PIC_TRACK_IDS)) CK(cudaMemcpyAsync(id, S.id, b4, k, s));
    }
    if (tile_offset) {
        const int nt1 = sim->g.ntiles + 1;
        int64_t* d = on_device ? tile_offset : (int64_t*)sim->rho;  // rho is scratch here
        CK(launch_offsets_to_i64(S.off[sim->cur], nt1, d, s));
        if (!on_device) CK(cudaMemcpyAsync(tile_offset, d, 8 * (size_t)nt1, k, s));
    }
    return sync_status(sim);
}

int64_t pic_num_particles(const pic_sim* sim, int species) {
    if (!sim || species < 0 || species >= sim->cfg.n_species) return -1;
    return sim->sp[species].n;
}

int64_t pic_num_tiles(const pic_sim* sim) { return sim ? sim->g.ntiles : -1; }

pic_status pic_probe_bounded_wait(int arrive, int64_t limit_cycles, void* cuda_stream) {
    if (limit_cycles < 1 || limit_cycles > 4000000000LL) return PIC_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned* d = nullptr;
    if (cudaMalloc((void**)&d, sizeof(unsigned)) != cudaSuccess) return PIC_ENOMEM;
    unsigned h = 0;
    const bool ok = launch_probe_wait(arrive != 0, limit_cycles, d, s) == cudaSuccess &&
                    cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                    cudaStreamSynchronize(s) == cudaSuccess;
    cudaFree(d);
    if (!ok) return PIC_ECUDA;
    return (h & ST_TIMEOUT) ? PIC_ETIMEOUT : PIC_OK;
}

pic_status pic_diagnostics(pic_sim* sim, pic_diag* out) {
    if (!sim || !out) return PIC_EINVAL;
    sim->err.clear();
    const Geom& g = sim->g;
    cudaStream_t s = sim->stream;
    const size_t ncell = (size_t)g.nx * g.ny;
    CK(cudaMemsetAsync(sim->rho, 0, ncell * 8, s));
    const int32_t* offs[MAX_SPECIES];
    for (int k = 0; k < sim->cfg.n_species; ++k) offs[k] = sim->sp[k].off[sim->cur];
    CK(launch_rho(g, sim->sp, sim->cfg.n_species, offs, sim->rho, s));
    CK(cudaMemsetAsync(sim->dred, 0, 8 * sizeof(double), s));
    const bool cont = sim->rho_prev_step >= 0 && sim->rho_prev_step + 1 == sim->step;
    CK(launch_grid_residuals(g, sim->F[sim->cur], sim->J[1 - sim->cur], sim->rho,
                             cont ? sim->rho_prev : nullptr, sim->cfg.background, sim->dred, s));
    double red[3];
    CK(cudaMemcpyAsync(red, sim->dred, sizeof red, cudaMemcpyDeviceToHost, s));
    const long long n = sim->step;
    double he, hb, hk = NAN;
    CK(cudaMemcpyAsync(&he, sim->hist_e + (n & (HIST - 1)), 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hb, sim->hist_b + (n & (HIST - 1)), 8, cudaMemcpyDeviceToHost, s));
    if (n > 0)
        CK(cudaMemcpyAsync(&hk, sim->hist_k + ((n - 1) & (HIST - 1)), 8, cudaMemcpyDeviceToHost, s));
    DevState h;
    CK(cudaMemcpyAsync(&h, sim->st, sizeof h, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    memset(out, 0, sizeof *out);
    out->step = n;
    out->time = n * sim->cfg.dt;
    out->w_e = he;
    out->w_b = hb;
    out->w_k = hk;
    // the moving window's open box, removal and injection make the periodic
    // Gauss and continuity residuals meaningless: not reported
    out->gauss_max = sim->window ? NAN : red[0];
    out->continuity_max = (cont && !sim->window) ? red[1] : NAN;
    out->charge_total = red[2];
    out->window_moves = sim->window ? h.win_moves : 0;
    long long lv = 0;
    for (int k = 0; k < sim->cfg.n_species; ++k) {
        if (sim->window) sim->sp[k].n = h.np[k];
        out->n_particles[k] = sim->sp[k].n;
        lv += h.leavers_sp[k];
    }
    out->leavers = n > 0 ? lv : 0;
    out->status_bits = h.status;
    std::swap(sim->rho, sim->rho_prev);
    sim->rho_prev_step = n;
    return status_from_bits(sim, h.status);
}

pic_status pic_get_history(pic_sim* sim, int64_t first, int64_t count, double* w_e, double* w_b,
                           double* w_k) {
    if (!sim || count < 0) return PIC_EINVAL;
    sim->err.clear();
    std::vector<double> he(HIST), hb(HIST), hk(HIST);
    CK(cudaMemcpyAsync(he.data(), sim->hist_e, HIST * 8, cudaMemcpyDeviceToHost, sim->stream));
    CK(cudaMemcpyAsync(hb.data(), sim->hist_b, HIST * 8, cudaMemcpyDeviceToHost, sim->stream));
    CK(cudaMemcpyAsync(hk.data(), sim->hist_k, HIST * 8, cudaMemcpyDeviceToHost, sim->stream));
    CK(cudaStreamSynchronize(sim->stream));
    const long long n = sim->step;
    for (int64_t k = 0; k < count; ++k) {
        const long long lev = first + k;
        const bool fld_ok = lev >= 0 && lev <= n && lev > n - HIST;
        const bool kin_ok = lev >= 0 && lev < n && lev > n - HIST;
        if (w_e) w_e[k] = fld_ok ? he[lev & (HIST - 1)] : NAN;
        if (w_b) w_b[k] = fld_ok ? hb[lev & (HIST - 1)] : NAN;
        if (w_k) w_k[k] = kin_ok ? hk[lev & (HIST - 1)] : NAN;
    }
    return PIC_OK;
}

pic_status pic_set_moving_window(pic_sim* sim, const pic_inject* inject) {
    if (!sim) return PIC_EINVAL;
    sim->err.clear();
    if (sim->batch) return fail(sim, PIC_EINVAL, "a batch member cannot have a moving window");
    if (sim->jfilter)
        return fail(sim, PIC_EINVAL, "the current filters are periodic: not with the moving window");
    for (int k = 0; k < sim->cfg.n_species; ++k)
        if (sim->sp[k].n > 0)
            return fail(sim, PIC_EINVAL, "set the moving window before loading particles");
    for (int k = 0; inject && k < sim->cfg.n_species; ++k) {
        const pic_inject& q = inject[k];
        if (q.k < 0 || q.k > 64 || q.capacity < 0 || q.capacity > 0x7fffffffLL ||
            !std::isfinite(q.x_start) || !std::isfinite(q.ux) || !std::isfinite(q.uy) ||
            !std::isfinite(q.uz))
            return fail(sim, PIC_EINVAL, "bad injection parameters for species %d", k);
    }
    CK(cudaStreamSynchronize(sim->stream));
    sim->window = 1;
    sim->g.open_x = 1;
    for (int k = 0; k < sim->cfg.n_species; ++k) {
        SpeciesDev& S = sim->sp[k];
        const pic_inject* q = inject ? &inject[k] : nullptr;
        S.inj_k = q ? q->k : 0;
        S.inj_u[0] = q ? q->ux : 0.f;
        S.inj_u[1] = q ? q->uy : 0.f;
        S.inj_u[2] = q ? q->uz : 0.f;
        S.inj_x0 = q ? q->x_start : 0.0;
        S.want_cap = q ? q->capacity : 0;
    }
    for (int b = 0; b < 2; ++b) CK(launch_zero_x_guards(sim->g, sim->F[b], 6, sim->stream));
    CK(cudaMemsetAsync(&sim->st->win_moves, 0, sizeof(long long), sim->stream));
    CK(cudaMemsetAsync(&sim->st->win_shift, 0, sizeof(int), sim->stream));
    invalidate_graphs(sim);
    pic_status r = refresh_level_energy(sim);
    if (r != PIC_OK) return r;
    CK(cudaStreamSynchronize(sim->stream));
    return PIC_OK;
}

pic_status pic_add_laser(pic_sim* sim, const pic_laser* laser) {
    if (!sim || !laser) return PIC_EINVAL;
    sim->err.clear();
    const pic_laser& l = *laser;
    if (!(l.type == PIC_LASER_PLANE || l.type == PIC_LASER_GAUSSIAN) || !(l.fwhm > 0) ||
        !(l.omega0 > 0) || !std::isfinite(l.a0) || !std::isfinite(l.start) ||
        !std::isfinite(l.polarization) ||
        (l.type == PIC_LASER_GAUSSIAN &&
         (!(l.W0 > 0) || !std::isfinite(l.focus) || !std::isfinite(l.axis))))
        return fail(sim, PIC_EINVAL, "bad laser parameters");
    LaserDev d;
    d.type = l.type == PIC_LASER_GAUSSIAN ? 1 : 0;
    d.start = l.start;
    d.fwhm = l.fwhm;
    d.a0 = l.a0;
    d.omega0 = l.omega0;
    d.polarization = l.polarization;
    d.W0 = l.W0;
    d.focus = l.focus;
    d.axis = l.axis;
    CK(launch_add_laser(sim->g, sim->F[sim->cur], d, sim->st, sim->stream));
    sim->rho_prev_step = -1;
    pic_status r = refresh_level_energy(sim);
    if (r != PIC_OK) return r;
    CK(cudaStreamSynchronize(sim->stream));
    return sync_status(sim);
}

pic_status pic_sync(pic_sim* sim) {
    if (!sim) return PIC_EINVAL;
    pic_status r = refresh_counts(sim);
    if (r != PIC_OK) return r;
    return sync_status(sim);
}

pic_status pic_clear_status(pic_sim* sim) {
    if (!sim) return PIC_EINVAL;
    CK(cudaStreamSynchronize(sim->stream));
    CK(cudaMemsetAsync(&sim->st->status, 0, sizeof(unsigned), sim->stream));
    CK(cudaStreamSynchronize(sim->stream));
    sim->err.clear();
    return PIC_OK;
}

pic_status pic_timing_stages(pic_sim* sim, double stage_ms[3], int64_t* steps, int reset) {
    if (!sim) return PIC_EINVAL;
    CK(cudaStreamSynchronize(sim->stream));
    constexpr size_t K = pic_sim::kStepEvents;
    double tot[3] = {0.0, 0.0, 0.0};
    for (size_t k = 0; k < sim->ev_used; ++k)
        for (int st = 0; st < 3; ++st) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, sim->ev_pool[K * k + st], sim->ev_pool[K * k + st + 1]));
            tot[st] += ms;
        }
    if (stage_ms)
        for (int st = 0; st < 3; ++st) stage_ms[st] = tot[st];
    if (steps) *steps = (int64_t)sim->ev_used;
    if (reset) sim->ev_used = 0;
    return PIC_OK;
}

pic_status pic_timing(pic_sim* sim, double* advance_ms, int64_t* advance_launches, int reset) {
    double ms[3];
    const pic_status r = pic_timing_stages(sim, ms, advance_launches, reset);
    if (r == PIC_OK && advance_ms) *advance_ms = ms[0];
    return r;
}

int64_t pic_kernel_launches(const pic_sim* sim) { return sim ? sim->launches : -1; }

const char* pic_last_error(const pic_sim* sim) { return sim ? sim->err.c_str() : "null handle"; }

void pic_destroy(pic_sim* sim) {
    if (!sim) return;
    if (sim->batch) batch_forget(sim->batch, sim);
    if (sim->stream) cudaStreamSynchronize(sim->stream);
    invalidate_graphs(sim);
    if (sim->cap_stream) cudaStreamDestroy(sim->cap_stream);
    if (sim->side_stream) {
        cudaStreamSynchronize(sim->side_stream);
        cudaStreamDestroy(sim->side_stream);
    }
    if (sim->ev_fork) cudaEventDestroy(sim->ev_fork);
    if (sim->ev_join) cudaEventDestroy(sim->ev_join);
    for (int b = 0; b < 2; ++b) {
        dfree(sim->F[b]);
        dfree(sim->J[b]);
    }
    for (auto ev : sim->ev_placeholder)
        if (ev) cudaEventDestroy(ev);
    for (auto ev : sim->ev_pool) cudaEventDestroy(ev);
    dfree(sim->gtmp);
    dfree(sim->rho);
    dfree(sim->rho_prev);
    dfree(sim->hist_e);
    dfree(sim->hist_b);
    dfree(sim->hist_k);
    dfree(sim->dred);
    dfree(sim->st);
    for (int k = 0; k < sim->cfg.n_species; ++k) {
        SpeciesDev& s = sim->sp[k];
        free_species(s);
        free_tile_arrays(s);
        dfree(s.cursor);
    }
    delete sim;
}

}  // extern "C"
