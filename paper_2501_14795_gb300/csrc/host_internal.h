// Host-side internals shared by the single-simulation runtime (pic_host.cu)
// and the batch runtime and autotuner (pic_batch.cu).  Not part of the ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "pic.h"
#include "pic_internal.h"

struct pic_sim {
    pic_config cfg;
    pic::Geom g;
    cudaStream_t stream = nullptr;       // caller's stream: all work is ordered on it
    cudaStream_t cap_stream = nullptr;   // private stream used only to capture graphs
    // The field branch of a step (current filter, field advance) runs on a
    // private side stream beside the re-sort's eviction and fill: forked from
    // the caller's stream after the scan, joined back before the step ends.
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    pic::DevState* st = nullptr;
    float* F[2] = {nullptr, nullptr};  // E|B, ping-pong
    float* J[2] = {nullptr, nullptr};  // current, ping-pong
    CUtensorMap fmap[2];
    CUtensorMap ymapF[2], ymapJ[2];    // the field kernel's boxes of F[b] and J[b]
    float* gtmp = nullptr;             // 3*nx*ny staging for set/get
    double* rho = nullptr;             // nx*ny FP64 charge density (no background)
    double* rho_prev = nullptr;
    long long rho_prev_step = -1;
    double* hist_e = nullptr;
    double* hist_b = nullptr;
    double* hist_k = nullptr;
    double* dred = nullptr;            // small FP64 reduction outputs
    pic::SpeciesDev sp[pic::MAX_SPECIES];
    int cur = 0;                       // parity: F[cur], J[cur] current, off[cur] current
    long long step = 0;                // host mirror of the time level
    // graphs
    cudaGraph_t graph[2] = {nullptr, nullptr};  // kept alive: its nodes address the exec's
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    // timing (PIC_TIMING): four events per step on the caller's stream,
    // recorded before the particle advance, after it, after the re-sort's fill
    // and at the end of the step (after the join with the field branch)
    static constexpr int kStepEvents = 4;
    cudaGraphNode_t ev_node[2][kStepEvents] = {};
    cudaEvent_t ev_placeholder[kStepEvents] = {};
    std::vector<cudaEvent_t> ev_pool;  // kStepEvents per timed step
    size_t ev_used = 0;                // steps recorded since reset
    long long launches = 0;
    int launches_per_step = 0;
    std::string err;
    // graph generation: bumped whenever the kernels' parameters change (a
    // reload or re-tiling), so that batches capturing this member rebuild
    unsigned long long gen = 0;
    pic_batch* batch = nullptr;  // batch this member belongs to, if any
    // current filter applied to J[b] between the re-sort and the field
    // advance; returns the kernels it launched or -1 (message in sim->err)
    int (*jfilter)(void* ctx, pic_sim* sim, cudaStream_t s, int b) = nullptr;
    void* jfilter_ctx = nullptr;
    int binomial_passes = 0;  // the binomial filter's passes when it is the installed filter
    int window = 0;           // moving window on (box open along x)
};

namespace pic {
namespace host {

pic_status fail(pic_sim* s, pic_status code, const char* fmt, ...);
int chunks_per_tile(const pic_sim* sim);
PushParams push_params(const pic_sim* sim, int b);
SortParams sort_params(const pic_sim* sim, int b);
YeeParams yee_params(const pic_sim* sim, int b, int chunks);
pic_status status_from_bits(pic_sim* sim, unsigned bits);
pic_status read_state(pic_sim* sim, DevState* h);
pic_status sync_status(pic_sim* sim);
void invalidate_graphs(pic_sim* sim);
// a member being destroyed leaves its batch
void batch_forget(pic_batch* batch, pic_sim* sim);
// Change the tile size of a loaded simulation in place: the particles are
// re-sorted into the new tiles (device to device), the tile bookkeeping and the
// TMA descriptors are rebuilt and the next step's J buffer is cleared.
pic_status retile(pic_sim* sim, int tile);
// Moving window: copy the device particle counts into the host mirrors
// (synchronises); no-op for a fixed box.
pic_status refresh_counts(pic_sim* sim);
// The denoiser has the grid g.
bool denoiser_fits(const pic_denoiser* d, const Geom& g);
// The network in the current-filter slot of B simulations of one grid at
// once (their currents from the device table jtab): gathered into a dense
// batch, denoised in groups of at most the network's batch_max, restored and
// written back.  Kernel timeouts go to `status`.  Returns the kernels
// launched, or -1 with the message in *err.
int denoiser_batch_filter(pic_denoiser* d, float* const* jtab, int B, const Geom& g,
                          unsigned* status, cudaStream_t s, std::string* err);

}  // namespace host
}  // namespace pic

#define PIC_CK(sim, call)                                                                 \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return ::pic::host::fail(sim, e_ == cudaErrorMemoryAllocation ? PIC_ENOMEM   \
                                                                         : PIC_ECUDA,     \
                                     "%s failed: %s", #call, cudaGetErrorString(e_));     \
    } while (0)
