// Batch runtime and autotuner behind the C ABI of include/pic.h.
//
// A batch steps many independent simulations with one launch per stage: the
// particle advance of all members in one persistent launch per (tile size,
// threads) group over a work list of (member, tile, slice) items, the four
// re-sort kernels over the flattened tiles of all members, and the field
// advance over all members' field tiles.  The members' kernel parameters live
// in device arrays (one set per buffer parity); each parity's step is one
// captured CUDA graph.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "host_internal.h"

using namespace pic;
using namespace pic::host;

struct pic_batch {
    std::vector<pic_sim*> m;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    bool strict = false;
    bool fp32_j = false;
    // what the graphs were built for: members' parity at phase 0 and generation
    std::vector<int> cur0;
    std::vector<unsigned long long> gen;
    int phase = 0;
    // device parameter blocks, per phase
    PushParams* d_push[2] = {nullptr, nullptr};
    CUtensorMap* d_tmaps[2] = {nullptr, nullptr};
    SortParams* d_sort[2] = {nullptr, nullptr};
    YeeParams* d_yee[2] = {nullptr, nullptr};
    float** d_jtab[2] = {nullptr, nullptr};  // the members' current buffers, per phase
    pic_denoiser* den = nullptr;  // network in the members' current-filter slot, or none
    int4* d_items = nullptr;
    int* d_tile_start = nullptr;
    int* d_ytile_start = nullptr;
    int* d_next = nullptr;  // one work counter per push group
    struct Group {
        int T, threads, first, count;
    };
    std::vector<Group> groups;
    int total_tiles = 0, total_ytiles = 0, max_nsp = 0;
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    long long launches = 0;
    int launches_per_step = 0;
    bool dirty = false;  // a member left: rebuild before the next step
    std::string err;
};

namespace {

pic_status bfail(pic_batch* b, pic_status code, const std::string& msg) {
    if (b) b->err = msg;
    return code;
}

#define BCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bfail(batch, e_ == cudaErrorMemoryAllocation ? PIC_ENOMEM : PIC_ECUDA,   \
                         std::string(#call " failed: ") + cudaGetErrorString(e_));          \
    } while (0)

void free_device(pic_batch* b) {
    for (int p = 0; p < 2; ++p) {
        cudaFree(b->d_push[p]);
        cudaFree(b->d_tmaps[p]);
        cudaFree(b->d_sort[p]);
        cudaFree(b->d_yee[p]);
        cudaFree(b->d_jtab[p]);
        b->d_jtab[p] = nullptr;
        b->d_push[p] = nullptr;
        b->d_tmaps[p] = nullptr;
        b->d_sort[p] = nullptr;
        b->d_yee[p] = nullptr;
    }
    cudaFree(b->d_items);
    cudaFree(b->d_tile_start);
    cudaFree(b->d_ytile_start);
    cudaFree(b->d_next);
    b->d_items = nullptr;
    b->d_tile_start = b->d_ytile_start = b->d_next = nullptr;
}

void free_graphs(pic_batch* b) {
    for (int p = 0; p < 2; ++p) {
        if (b->gexec[p]) cudaGraphExecDestroy(b->gexec[p]);
        if (b->graph[p]) cudaGraphDestroy(b->graph[p]);
        b->gexec[p] = nullptr;
        b->graph[p] = nullptr;
    }
}

// Build the work list and the per-phase parameter arrays from the members'
// current state; phase 0 uses each member's present buffer parity.
pic_status prepare(pic_batch* batch) {
    cudaStream_t s = batch->stream;
    BCK(cudaStreamSynchronize(s));
    free_graphs(batch);
    free_device(batch);
    const int n = (int)batch->m.size();
    batch->cur0.resize(n);
    batch->gen.resize(n);
    std::vector<PushParams> hp[2];
    std::vector<CUtensorMap> ht[2];
    std::vector<SortParams> hs[2];
    std::vector<YeeParams> hy[2];
    std::vector<float*> hj[2];
    std::vector<int> tile_start(n + 1, 0), ytile_start(n + 1, 0);
    struct Item {
        int4 v;
        long long cost;
        int group;
    };
    std::vector<Item> items;
    std::map<std::pair<int, int>, int> gid;  // (T, threads) -> group
    batch->groups.clear();
    batch->max_nsp = 0;
    for (int k = 0; k < n; ++k) {
        pic_sim* sim = batch->m[k];
        batch->cur0[k] = sim->cur;
        batch->gen[k] = sim->gen;
        const int chunks = chunks_per_tile(sim);
        for (int p = 0; p < 2; ++p) {
            const int b = sim->cur ^ p;
            hp[p].push_back(push_params(sim, b));
            ht[p].push_back(sim->fmap[b]);
            hs[p].push_back(sort_params(sim, b));
            hy[p].push_back(yee_params(sim, b, chunks));
            hj[p].push_back(sim->J[b]);
        }
        tile_start[k + 1] = tile_start[k] + sim->g.ntiles;
        ytile_start[k + 1] = ytile_start[k] + yee_tiles(sim->g);
        batch->max_nsp = std::max(batch->max_nsp, sim->cfg.n_species);
        const auto key = std::make_pair(sim->g.T, sim->cfg.threads);
        auto it = gid.find(key);
        if (it == gid.end()) {
            it = gid.emplace(key, (int)batch->groups.size()).first;
            batch->groups.push_back({sim->g.T, sim->cfg.threads, 0, 0});
        }
        // cost of an item: the particles of its slice of the tile, all species
        int64_t per_tile = 0;
        for (int sp = 0; sp < sim->cfg.n_species; ++sp)
            per_tile += sim->g.ntiles ? sim->sp[sp].n / sim->g.ntiles : 0;
        const long long cost = per_tile / chunks + 1;
        for (int t = 0; t < sim->g.ntiles; ++t)
            for (int c = 0; c < chunks; ++c) items.push_back({make_int4(k, t, c, 0), cost, it->second});
    }
    if (tile_start[n] > 0x7fffffff / 8 || (long long)items.size() > 0x7fffffff)
        return bfail(batch, PIC_EINVAL, "batch too large");
    // group items, costliest first inside a group (stable: tile order otherwise)
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) {
        if (a.group != b.group) return a.group < b.group;
        return a.cost > b.cost;
    });
    std::vector<int4> hv(items.size());
    for (size_t i = 0; i < items.size(); ++i) {
        hv[i] = items[i].v;
        auto& g = batch->groups[items[i].group];
        if (g.count == 0) g.first = (int)i;
        g.count += 1;
    }
    batch->total_tiles = tile_start[n];
    batch->total_ytiles = ytile_start[n];
    auto up = [&](auto** dst, const auto& src) -> cudaError_t {
        using T = std::remove_reference_t<decltype(**dst)>;
        cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * std::max<size_t>(src.size(), 1));
        if (e != cudaSuccess) return e;
        if (src.empty()) return cudaSuccess;
        return cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s);
    };
    for (int p = 0; p < 2; ++p) {
        BCK(up(&batch->d_push[p], hp[p]));
        BCK(up(&batch->d_tmaps[p], ht[p]));
        BCK(up(&batch->d_sort[p], hs[p]));
        BCK(up(&batch->d_yee[p], hy[p]));
        BCK(up(&batch->d_jtab[p], hj[p]));
    }
    BCK(up(&batch->d_items, hv));
    BCK(up(&batch->d_tile_start, tile_start));
    BCK(up(&batch->d_ytile_start, ytile_start));
    BCK(cudaMalloc((void**)&batch->d_next, sizeof(int) * std::max<size_t>(batch->groups.size(), 1)));
    BCK(cudaStreamSynchronize(s));
    batch->phase = 0;
    batch->dirty = false;
    return PIC_OK;
}

// Enqueue one batched step of phase p; returns kernels launched or -1.
int enqueue_batch_step(pic_batch* batch, cudaStream_t s, int p) {
    cudaError_t e = cudaSuccess;
    int n = 0;
    const int ng = (int)batch->groups.size();
    if (ng > 0) e = cudaMemsetAsync(batch->d_next, 0, sizeof(int) * ng, s);
    for (int gi = 0; gi < ng && e == cudaSuccess; ++gi) {
        const auto& g = batch->groups[gi];
        PushBatch pb;
        pb.members = batch->d_push[p];
        pb.tmaps = batch->d_tmaps[p];
        pb.items = batch->d_items + g.first;
        pb.nitems = g.count;
        pb.next = batch->d_next + gi;
        pb.fp32_j = batch->fp32_j ? 1 : 0;
        e = batch->strict ? launch_push_batch_strict(pb, g.T, g.threads, 0, s)
                          : launch_push_batch_fast(pb, g.T, g.threads, 0, s);
        n += g.count > 0;
    }
    if (e == cudaSuccess) {
        SortBatch sb;
        sb.members = batch->d_sort[p];
        sb.tile_start = batch->d_tile_start;
        sb.nmembers = (int)batch->m.size();
        sb.total_tiles = batch->total_tiles;
        sb.max_nsp = batch->max_nsp;
        e = launch_sort_batch(sb, s);
        n += sb.total_tiles > 0 ? 4 : 1;
    }
    if (e == cudaSuccess && batch->den) {
        // the current-filter slot: after the deposit and the re-sort, before
        // the field advance, all members' currents through the network at once
        std::string why;
        const int k = denoiser_batch_filter(batch->den, batch->d_jtab[p], (int)batch->m.size(),
                                            batch->m[0]->g, &batch->m[0]->st->status, s, &why);
        if (k < 0) {
            batch->err = why;
            return -1;
        }
        n += k;
    }
    if (e == cudaSuccess) {
        YeeBatch yb;
        yb.members = batch->d_yee[p];
        yb.ytile_start = batch->d_ytile_start;
        yb.nmembers = (int)batch->m.size();
        yb.total_ytiles = batch->total_ytiles;
        e = launch_yee_batch(yb, s);
        n += yb.total_ytiles > 0;
    }
    if (e != cudaSuccess) {
        batch->err = std::string("batched launch failed: ") + cudaGetErrorString(e);
        return -1;
    }
    return n;
}

pic_status build_batch_graph(pic_batch* batch, int p) {
    cudaGraph_t graph = nullptr;
    BCK(cudaStreamBeginCapture(batch->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int n = enqueue_batch_step(batch, batch->cap_stream, p);
    cudaError_t e = cudaStreamEndCapture(batch->cap_stream, &graph);
    if (n < 0) {
        if (graph) cudaGraphDestroy(graph);
        return PIC_ECUDA;
    }
    BCK(e);
    batch->launches_per_step = n;
    e = cudaGraphInstantiate(&batch->gexec[p], graph, 0);
    batch->graph[p] = graph;
    BCK(e);
    return PIC_OK;
}

bool stale(const pic_batch* batch) {
    if (batch->dirty) return true;
    for (size_t k = 0; k < batch->m.size(); ++k) {
        const pic_sim* sim = batch->m[k];
        if (sim->gen != batch->gen[k] || sim->cur != (batch->cur0[k] ^ batch->phase)) return true;
    }
    return false;
}

// ---------------------------------------------------------------- autotuner
struct TuneKey {
    int nx, ny, nsp;
    long long ppc_milli;  // total particles per cell x 1000
    int strict, device;  // strict: the PIC_STRICT_FP | PIC_FP32_J bits (other kernels)
    bool operator<(const TuneKey& o) const {
        return std::tie(nx, ny, nsp, ppc_milli, strict, device) <
               std::tie(o.nx, o.ny, o.nsp, o.ppc_milli, o.strict, o.device);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;

// Saved state of a simulation: particles (in the main arrays' layout), E|B of
// the current level, the last J, the energy history and the device status.
struct Snapshot {
    struct Sp {
        int32_t *ix = nullptr, *iy = nullptr, *id = nullptr;
        float *x = nullptr, *y = nullptr, *ux = nullptr, *uy = nullptr, *uz = nullptr;
        int64_t n = 0;
    } sp[MAX_SPECIES];
    float *F = nullptr, *J = nullptr;
    double* hist = nullptr;
    DevState st;
    int cur = 0;
    long long step = 0, rho_prev_step = -1;
    void release() {
        for (auto& s : sp) {
            void* p[] = {s.ix, s.iy, s.id, s.x, s.y, s.ux, s.uy, s.uz};
            for (void* q : p) cudaFree(q);
            s = Sp();
        }
        cudaFree(F);
        cudaFree(J);
        cudaFree(hist);
        F = J = nullptr;
        hist = nullptr;
    }
};

pic_status save(pic_sim* sim, Snapshot& S) {
    cudaStream_t s = sim->stream;
    const bool track = (sim->cfg.flags & PIC_TRACK_IDS) != 0;
    for (int k = 0; k < sim->cfg.n_species; ++k) {
        const SpeciesDev& D = sim->sp[k];
        auto& o = S.sp[k];
        o.n = D.n;
        if (D.n == 0) continue;
        const size_t b4 = 4 * (size_t)D.n;
        PIC_CK(sim, cudaMalloc((void**)&o.ix, b4));
        PIC_CK(sim, cudaMalloc((void**)&o.iy, b4));
        PIC_CK(sim, cudaMalloc((void**)&o.x, b4));
        PIC_CK(sim, cudaMalloc((void**)&o.y, b4));
        PIC_CK(sim, cudaMalloc((void**)&o.ux, b4));
        PIC_CK(sim, cudaMalloc((void**)&o.uy, b4));
        PIC_CK(sim, cudaMalloc((void**)&o.uz, b4));
        if (track) PIC_CK(sim, cudaMalloc((void**)&o.id, b4));
    }
    for (int k = 0; k < sim->cfg.n_species; ++k) {
        pic_status r = pic_get_particles(sim, k, S.sp[k].ix, S.sp[k].iy, S.sp[k].x, S.sp[k].y,
                                         S.sp[k].ux, S.sp[k].uy, S.sp[k].uz, S.sp[k].id, nullptr,
                                         1);
        if (r != PIC_OK) return r;
    }
    const size_t fb = 6 * (size_t)sim->g.cstride * 4, jb = 3 * (size_t)sim->g.cstride * 4;
    PIC_CK(sim, cudaMalloc((void**)&S.F, fb));
    PIC_CK(sim, cudaMalloc((void**)&S.J, jb));
    PIC_CK(sim, cudaMalloc((void**)&S.hist, 3 * HIST * sizeof(double)));
    PIC_CK(sim, cudaMemcpyAsync(S.F, sim->F[sim->cur], fb, cudaMemcpyDeviceToDevice, s));
    PIC_CK(sim, cudaMemcpyAsync(S.J, sim->J[1 - sim->cur], jb, cudaMemcpyDeviceToDevice, s));
    PIC_CK(sim, cudaMemcpyAsync(S.hist, sim->hist_e, HIST * 8, cudaMemcpyDeviceToDevice, s));
    PIC_CK(sim, cudaMemcpyAsync(S.hist + HIST, sim->hist_b, HIST * 8, cudaMemcpyDeviceToDevice, s));
    PIC_CK(sim, cudaMemcpyAsync(S.hist + 2 * HIST, sim->hist_k, HIST * 8, cudaMemcpyDeviceToDevice, s));
    pic_status r = read_state(sim, &S.st);
    S.cur = sim->cur;
    S.step = sim->step;
    S.rho_prev_step = sim->rho_prev_step;
    return r;
}

pic_status restore(pic_sim* sim, const Snapshot& S) {
    cudaStream_t s = sim->stream;
    // the fields go back into the parity the snapshot was taken at
    sim->cur = S.cur;
    sim->step = S.step;
    const size_t fb = 6 * (size_t)sim->g.cstride * 4, jb = 3 * (size_t)sim->g.cstride * 4;
    PIC_CK(sim, cudaMemcpyAsync(sim->F[sim->cur], S.F, fb, cudaMemcpyDeviceToDevice, s));
    PIC_CK(sim, cudaMemcpyAsync(sim->J[1 - sim->cur], S.J, jb, cudaMemcpyDeviceToDevice, s));
    // the next step deposits into J[cur]: clear it whatever the tuning steps left
    PIC_CK(sim, cudaMemsetAsync(sim->J[sim->cur], 0, jb, s));
    PIC_CK(sim, cudaMemcpyAsync(sim->hist_e, S.hist, HIST * 8, cudaMemcpyDeviceToDevice, s));
    PIC_CK(sim, cudaMemcpyAsync(sim->hist_b, S.hist + HIST, HIST * 8, cudaMemcpyDeviceToDevice, s));
    PIC_CK(sim, cudaMemcpyAsync(sim->hist_k, S.hist + 2 * HIST, HIST * 8, cudaMemcpyDeviceToDevice, s));
    for (int k = 0; k < sim->cfg.n_species; ++k) {
        const auto& o = S.sp[k];
        // the load replaces the particles and re-primes the level's energy;
        // the saved history is copied again afterwards
        pic_status r = pic_load_particles(sim, k, o.n, o.ix, o.iy, o.x, o.y, o.ux, o.uy, o.uz,
                                          o.id, 1);
        if (r != PIC_OK) return r;
    }
    PIC_CK(sim, cudaMemcpyAsync(sim->hist_e, S.hist, HIST * 8, cudaMemcpyDeviceToDevice, s));
    PIC_CK(sim, cudaMemcpyAsync(sim->hist_b, S.hist + HIST, HIST * 8, cudaMemcpyDeviceToDevice, s));
    PIC_CK(sim, cudaMemcpyAsync(sim->hist_k, S.hist + 2 * HIST, HIST * 8, cudaMemcpyDeviceToDevice, s));
    PIC_CK(sim, cudaMemcpyAsync(sim->st, &S.st, sizeof(DevState), cudaMemcpyHostToDevice, s));
    PIC_CK(sim, cudaStreamSynchronize(s));
    sim->rho_prev_step = S.rho_prev_step;
    return PIC_OK;
}

// mean step time of the simulation as it is configured now
pic_status time_steps(pic_sim* sim, int steps, double* ms) {
    pic_status r = pic_step(sim, 2);  // warm-up; builds both parities' graphs
    if (r != PIC_OK) return r;
    cudaEvent_t a = nullptr, b = nullptr;
    PIC_CK(sim, cudaEventCreate(&a));
    cudaError_t e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        PIC_CK(sim, e);
    }
    e = cudaEventRecord(a, sim->stream);
    if (e == cudaSuccess) r = pic_step(sim, steps);
    if (e == cudaSuccess && r == PIC_OK) e = cudaEventRecord(b, sim->stream);
    if (e == cudaSuccess && r == PIC_OK) e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess && r == PIC_OK) e = cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (r != PIC_OK) return r;
    PIC_CK(sim, e);
    *ms = t / steps;
    return sync_status(sim);
}

}  // namespace

namespace pic {
namespace host {

void batch_forget(pic_batch* batch, pic_sim* sim) {
    if (batch->stream) cudaStreamSynchronize(batch->stream);
    auto it = std::find(batch->m.begin(), batch->m.end(), sim);
    if (it == batch->m.end()) return;
    batch->m.erase(it);
    free_graphs(batch);
    batch->dirty = true;
}

}  // namespace host
}  // namespace pic

extern "C" {

pic_status pic_set_tiling(pic_sim* sim, int tile, int threads) {
    if (!sim) return PIC_EINVAL;
    sim->err.clear();
    if (threads != 0 && (threads < 64 || threads > 512 || threads % 32))
        return fail(sim, PIC_EINVAL, "threads %d not in 64..512 or not a multiple of 32", threads);
    pic_status r = retile(sim, tile);
    if (r != PIC_OK) return r;
    if (threads > 0 && threads != sim->cfg.threads) {
        sim->cfg.threads = threads;
        invalidate_graphs(sim);
    }
    return PIC_OK;
}

pic_status pic_autotune(pic_sim* sim, int steps, int force, int* tile, int* threads,
                        double* step_ms) {
    if (!sim) return PIC_EINVAL;
    sim->err.clear();
    if (steps < 1) return fail(sim, PIC_EINVAL, "steps must be >= 1");
    {
        pic_status r = refresh_counts(sim);
        if (r != PIC_OK) return r;
    }
    int dev = 0;
    PIC_CK(sim, cudaGetDevice(&dev));
    // particles per cell as loaded (all species)
    double ppc = 0.0;
    for (int k = 0; k < sim->cfg.n_species; ++k)
        ppc += (double)sim->sp[k].n / ((double)sim->cfg.nx * sim->cfg.ny);
    const TuneKey key{sim->cfg.nx, sim->cfg.ny, sim->cfg.n_species, std::llround(ppc * 1000.0),
                      (int)(sim->cfg.flags & (PIC_STRICT_FP | PIC_FP32_J)), dev};
    if (!force) {
        std::pair<int, int> hit{0, 0};
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) hit = it->second;
        }
        if (hit.first) {
            pic_status r = pic_set_tiling(sim, hit.first, hit.second);
            if (r != PIC_OK) return r;
            if (tile) *tile = hit.first;
            if (threads) *threads = hit.second;
            if (step_ms) *step_ms = 0.0;
            return PIC_OK;
        }
    }
    pic_status r = sync_status(sim);
    if (r != PIC_OK) return r;
    Snapshot snap;
    r = save(sim, snap);
    if (r != PIC_OK) {
        snap.release();
        return r;
    }
    const int tiles[3] = {8, 16, 32};
    const int thr[4] = {64, 128, 256, 512};
    int best_t = sim->cfg.tile, best_n = sim->cfg.threads;
    double best = INFINITY;
    for (int T : tiles) {
        if (sim->cfg.nx % T || sim->cfg.ny % T) continue;
        for (int n : thr) {
            r = pic_set_tiling(sim, T, n);
            if (r == PIC_OK) {
                double ms = 0.0;
                r = time_steps(sim, steps, &ms);
                if (r == PIC_OK && ms < best) {
                    best = ms;
                    best_t = T;
                    best_n = n;
                }
            }
            // every candidate starts from the saved state
            const std::string why = sim->err;
            pic_status r2 = restore(sim, snap);
            if (r != PIC_OK || r2 != PIC_OK) {
                snap.release();
                if (r != PIC_OK)
                    fail(sim, r, "autotune candidate T=%d threads=%d: %s", T, n, why.c_str());
                return r != PIC_OK ? r : r2;
            }
        }
    }
    r = pic_set_tiling(sim, best_t, best_n);
    if (r == PIC_OK) r = restore(sim, snap);
    snap.release();
    if (r != PIC_OK) return r;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = {best_t, best_n};
    }
    if (tile) *tile = best_t;
    if (threads) *threads = best_n;
    if (step_ms) *step_ms = best;
    return PIC_OK;
}

pic_status pic_init_batch(const pic_config* cfgs, int n, void* cuda_stream, pic_sim** out) {
    if (!out || !cfgs || n < 0) return PIC_EINVAL;
    for (int k = 0; k < n; ++k) out[k] = nullptr;
    for (int k = 0; k < n; ++k) {
        pic_status r = pic_init(cfgs + k, cuda_stream, out + k);
        if (r != PIC_OK) {
            for (int j = 0; j < k; ++j) {
                pic_destroy(out[j]);
                out[j] = nullptr;
            }
            return r;
        }
    }
    return PIC_OK;
}

pic_status pic_batch_create(pic_sim* const* members, int n, void* cuda_stream, pic_batch** out) {
    if (!out) return PIC_EINVAL;
    *out = nullptr;
    if (!members || n < 1) return PIC_EINVAL;
    pic_batch* batch = new pic_batch();
    batch->stream = (cudaStream_t)cuda_stream;
    for (int k = 0; k < n; ++k) {
        pic_sim* sim = members[k];
        std::string why;
        if (!sim) why = "null member";
        else if (sim->batch) why = "member already belongs to a batch";
        else if (sim->stream != batch->stream) why = "member created on another stream";
        else if (std::find(batch->m.begin(), batch->m.end(), sim) != batch->m.end())
            why = "member listed twice";
        else if (k > 0 && ((sim->cfg.flags ^ members[0]->cfg.flags) & PIC_STRICT_FP))
            why = "members differ in PIC_STRICT_FP";
        else if (k > 0 && ((sim->cfg.flags ^ members[0]->cfg.flags) & PIC_FP32_J))
            why = "members differ in PIC_FP32_J";
        else if (sim->jfilter)
            why = "member has a current filter installed";
        else if (sim->window)
            why = "member has a moving window";
        if (!why.empty()) {
            if (sim) fail(sim, PIC_EINVAL, "pic_batch_create: %s", why.c_str());
            delete batch;
            return PIC_EINVAL;
        }
        batch->m.push_back(sim);
    }
    batch->strict = (members[0]->cfg.flags & PIC_STRICT_FP) != 0;
    batch->fp32_j = (members[0]->cfg.flags & PIC_FP32_J) != 0;
    if (cudaStreamCreateWithFlags(&batch->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete batch;
        return PIC_ECUDA;
    }
    for (pic_sim* sim : batch->m) {
        pic_status r = sync_status(sim);
        if (r != PIC_OK) {
            pic_batch_destroy(batch);
            return r;
        }
        sim->batch = batch;
    }
    pic_status r = prepare(batch);
    if (r != PIC_OK) {
        pic_batch_destroy(batch);
        return r;
    }
    *out = batch;
    return PIC_OK;
}

pic_status pic_batch_set_denoiser(pic_batch* batch, pic_denoiser* d) {
    if (!batch) return PIC_EINVAL;
    batch->err.clear();
    if (d)
        for (size_t k = 0; k < batch->m.size(); ++k) {
            const Geom& g = batch->m[k]->g;
            const Geom& g0 = batch->m[0]->g;
            if (!denoiser_fits(d, g) || g.P != g0.P || g.cstride != g0.cstride)
                return bfail(batch, PIC_EINVAL,
                             "pic_batch_set_denoiser: member " + std::to_string(k) +
                                 " does not have the network's grid");
        }
    BCK(cudaStreamSynchronize(batch->stream));
    batch->den = d;
    free_graphs(batch);
    return PIC_OK;
}

pic_status pic_batch_step(pic_batch* batch, int nsteps) {
    if (!batch) return PIC_EINVAL;
    if (nsteps < 0) return bfail(batch, PIC_EINVAL, "negative step count");
    batch->err.clear();
    if (batch->m.empty()) return PIC_OK;
    for (pic_sim* sim : batch->m) {
        if (sim->jfilter)
            return bfail(batch, PIC_EINVAL, "a member has a current filter installed");
        if (sim->window) return bfail(batch, PIC_EINVAL, "a member has a moving window");
    }
    for (int k = 0; k < nsteps; ++k) {
        if (stale(batch)) {
            pic_status r = prepare(batch);
            if (r != PIC_OK) return r;
        }
        const int p = batch->phase;
        if (!batch->gexec[p]) {
            pic_status r = build_batch_graph(batch, p);
            if (r != PIC_OK) return r;
        }
        BCK(cudaGraphLaunch(batch->gexec[p], batch->stream));
        batch->launches += batch->launches_per_step;
        for (pic_sim* sim : batch->m) {
            sim->cur ^= 1;
            sim->step += 1;
        }
        batch->phase ^= 1;
    }
    return PIC_OK;
}

pic_status pic_batch_sync(pic_batch* batch, int* member) {
    if (member) *member = -1;
    if (!batch) return PIC_EINVAL;
    BCK(cudaStreamSynchronize(batch->stream));
    for (size_t k = 0; k < batch->m.size(); ++k) {
        pic_status r = sync_status(batch->m[k]);
        if (r != PIC_OK) {
            if (member) *member = (int)k;
            batch->err = std::string("member ") + std::to_string(k) + ": " + batch->m[k]->err;
            return r;
        }
    }
    return PIC_OK;
}

int64_t pic_batch_kernel_launches(const pic_batch* batch, int* per_step) {
    if (!batch) return -1;
    if (per_step) *per_step = batch->launches_per_step;
    return batch->launches;
}

const char* pic_batch_last_error(const pic_batch* batch) {
    return batch ? batch->err.c_str() : "null handle";
}

void pic_batch_destroy(pic_batch* batch) {
    if (!batch) return;
    if (batch->stream) cudaStreamSynchronize(batch->stream);
    free_graphs(batch);
    free_device(batch);
    if (batch->cap_stream) cudaStreamDestroy(batch->cap_stream);
    for (pic_sim* sim : batch->m)
        if (sim && sim->batch == batch) sim->batch = nullptr;
    delete batch;
}

}  // extern "C"
