// pic_tile_sort_noalloc: sorting particles into tiles without allocating.
//
// Some callers cannot call cudaMalloc: code running inside a host callback or
// a custom allocator's hook, plugins whose host application owns every device
// allocation and forbids others, or a process that has carved all device
// memory into its own pool up front.  For them this entry point sorts
// caller-owned particle arrays into caller-owned output arrays by tile, the
// same counting sort pic_load_particles performs, with its scratch (the
// per-tile counters and cursors and a validation counter) in the fixed
// device array below instead of memory allocated per call.  It calls no
// cudaMalloc, no cudaFree and no allocating library routine.
//
// The array is file-scope `static __device__`: every GPU that loads this
// library holds its 256 KB + 256 B until the process exits, and every call
// on a device shares it.  Host code may not use the array's name as a device
// address (in host code it names a host-side stand-in), so every call looks
// up the device address with cudaGetSymbolAddress, with the caller's device
// current, and checks the result; the address is not cached, so a device
// reset between calls (which reloads the module and may move the array) is
// harmless.  Each call clears the counters it uses before using them.  Each
// call synchronises its stream (it reads the validation counter back before
// scanning), so it cannot be made during a stream capture.  Two calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on the shared array and give wrong results: serialise them.
#include <cuda_runtime.h>

#include "pic.h"
#include "device_util.cuh"

namespace {

constexpr int kMaxTiles = PIC_NOALLOC_MAX_TILES;
constexpr int kBadSlot = kMaxTiles;  // validation-failure counter after the tile counters
constexpr int kScratchInts = kMaxTiles + 64;
static __device__ __align__(256) int32_t g_scratch[kScratchInts];

// Device address of g_scratch and the SM count of the current device.
cudaError_t scratch_address(int32_t** out, int* sms) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *out = static_cast<int32_t*>(p);
    return cudaSuccess;
}

struct In {
    const int32_t *ix, *iy;
    const float *x, *y, *ux, *uy, *uz;
};
struct Out {
    int32_t *ix, *iy;
    float *x, *y, *ux, *uy, *uz;
    int64_t* off;
};

__device__ __forceinline__ bool valid(const In& a, int k, int nx, int ny) {
    return a.ix[k] >= 0 && a.ix[k] < nx && a.iy[k] >= 0 && a.iy[k] < ny && a.x[k] >= 0.f &&
           a.x[k] < 1.f && a.y[k] >= 0.f && a.y[k] < 1.f && isfinite(a.ux[k]) &&
           isfinite(a.uy[k]) && isfinite(a.uz[k]);
}

__global__ void k_na_count(In a, int n, int nx, int ny, int T, int ntx, int32_t* scratch) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if (!valid(a, k, nx, ny)) {
            atomicAdd(&scratch[kBadSlot], 1);
            continue;
        }
        atomicAdd(&scratch[(a.iy[k] / T) * ntx + a.ix[k] / T], 1);
    }
}

// exclusive scan of the counts into the caller's int64 bookmarks; the counts
// are cleared behind it so that they serve as the scatter cursors
__global__ void __launch_bounds__(1024) k_na_scan(int nt, int64_t* off, int32_t* scratch) {
    __shared__ long long sWarp[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int per = (nt + 1023) / 1024;
    const int t0 = min(tid * per, nt), t1 = min(t0 + per, nt);
    long long mine = 0;
    for (int t = t0; t < t1; ++t) mine += scratch[t];
    long long incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) sWarp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const long long w = sWarp[lane];
        long long wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const long long v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        sWarp[lane] = wi - w;
    }
    __syncthreads();
    long long run = sWarp[wid] + incl - mine;
    for (int t = t0; t < t1; ++t) {
        const int c = scratch[t];
        off[t] = run;
        scratch[t] = 0;
        run += c;
    }
    if (tid == 1023) off[nt] = run;
}

__global__ void k_na_scatter(In a, Out b, int n, int T, int ntx, int32_t* scratch) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int t = (a.iy[k] / T) * ntx + a.ix[k] / T;
        const long long p = b.off[t] + atomicAdd(&scratch[t], 1);
        b.ix[p] = a.ix[k];
        b.iy[p] = a.iy[k];
        b.x[p] = a.x[k];
        b.y[p] = a.y[k];
        b.ux[p] = a.ux[k];
        b.uy[p] = a.uy[k];
        b.uz[p] = a.uz[k];
    }
}

}  // namespace

extern "C" pic_status pic_tile_sort_noalloc(int nx, int ny, int tile, int64_t n,
                                            const int32_t* ix, const int32_t* iy, const float* x,
                                            const float* y, const float* ux, const float* uy,
                                            const float* uz, int32_t* ix_out, int32_t* iy_out,
                                            float* x_out, float* y_out, float* ux_out,
                                            float* uy_out, float* uz_out, int64_t* tile_offset,
                                            void* cuda_stream) {
    if (!(tile == 8 || tile == 16 || tile == 32) || nx < tile || ny < tile || nx % tile ||
        ny % tile || nx > 32768 || ny > 32768 || n < 0 || n > 0x7fffffffLL || !tile_offset)
        return PIC_EINVAL;
    const long long ntiles = (long long)(nx / tile) * (ny / tile);
    if (ntiles > kMaxTiles) return PIC_EINVAL;  // beyond the fixed scratch array
    if (n > 0 && (!ix || !iy || !x || !y || !ux || !uy || !uz || !ix_out || !iy_out || !x_out ||
                  !y_out || !ux_out || !uy_out || !uz_out))
        return PIC_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int32_t* scratch = nullptr;
    int sms = 0;
    if (scratch_address(&scratch, &sms) != cudaSuccess) return PIC_ECUDA;
    const int nn = static_cast<int>(n), ntx = nx / tile;
    const In a{ix, iy, x, y, ux, uy, uz};
    const Out b{ix_out, iy_out, x_out, y_out, ux_out, uy_out, uz_out, tile_offset};
    int blocks = (nn + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (sms < 1) sms = 1;
    if (blocks > sms * 16) blocks = sms * 16;  // grid-stride loops beyond this
    // clear the counters and the validation counter left by the previous call
    if (cudaMemsetAsync(scratch, 0, sizeof(int32_t) * ntiles, s) != cudaSuccess ||
        cudaMemsetAsync(scratch + kBadSlot, 0, sizeof(int32_t), s) != cudaSuccess)
        return PIC_ECUDA;
    if (nn > 0) k_na_count<<<blocks, 256, 0, s>>>(a, nn, nx, ny, tile, ntx, scratch);
    int32_t bad = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&bad, scratch + kBadSlot, sizeof bad, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PIC_ECUDA;
    if (bad) return PIC_EINVAL;  // a cell outside the grid, an offset outside [0,1) or a NaN/inf
    k_na_scan<<<1, 1024, 0, s>>>(static_cast<int>(ntiles), tile_offset, scratch);
    if (nn > 0) k_na_scatter<<<blocks, 256, 0, s>>>(a, b, nn, tile, ntx, scratch);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return PIC_ECUDA;
    return PIC_OK;
}
