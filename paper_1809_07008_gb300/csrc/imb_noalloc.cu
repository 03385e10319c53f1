// imb_noalloc.cu -- particle-to-bin map that allocates no device memory.
//
// Some callers cannot call cudaMalloc: hosts that hand every byte of device memory
// to their own pool, or real-time loops that must not touch the allocator.  imb_bin_particles_noalloc
// gives them the binning step of the particle map with inputs and outputs in their
// own device buffers; its scratch (per-bin counts and fill cursors) lives in the
// fixed array below, which every GPU that loads the library holds until exit.
#include <mutex>

#include "../../include/imblbm.h"
#include "imb_device.cuh"

namespace {

constexpr int MAX_BINS = IMB_NOALLOC_MAX_BINS;

// [0, MAX_BINS): counts, [MAX_BINS, 2 MAX_BINS): fill cursors.  Shared by every call.
static __device__ __align__(256) int g_bin_scratch[2 * MAX_BINS];

// Device address of g_bin_scratch per device, looked up once with that device current.
constexpr int MAX_DEVICES = 64;
int *g_scratch_ptr[MAX_DEVICES] = {};
std::mutex g_scratch_mutex;

__device__ __forceinline__ int bin_index(double px, double py, int nbx, int nby) {
    int bx = (int)floor(px / (double)imb::TILE), by = (int)floor(py / (double)imb::TILE);
    bx = bx < 0 ? 0 : (bx >= nbx ? nbx - 1 : bx);
    by = by < 0 ? 0 : (by >= nby ? nby - 1 : by);
    return by * nbx + bx;
}

__global__ void k_na_clear(int *scratch, int nbins) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
        scratch[b] = 0;
        scratch[MAX_BINS + b] = 0;
    }
}

__global__ void k_na_count(const double *__restrict__ x, int n, int nbx, int nby, int *scratch) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        atomicAdd(&scratch[bin_index(x[2 * p], x[2 * p + 1], nbx, nby)], 1);
}

// exclusive scan of the counts into bin_start[0..nbins] (one block)
__global__ void __launch_bounds__(1024) k_na_scan(const int *scratch, int *bin_start, int nbins) {
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (nbins + 1023) / 1024;
    const int b0 = min((int)threadIdx.x * per, nbins), b1 = min(b0 + per, nbins);
    int tot = 0;
    for (int b = b0; b < b1; ++b) tot += scratch[b];
    int incl = tot;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int run = (warp ? wsum[warp - 1] : 0) + incl - tot;
    for (int b = b0; b < b1; ++b) {
        bin_start[b] = run;
        run += scratch[b];
    }
    if (threadIdx.x == 1023) bin_start[nbins] = wsum[31];
}

__global__ void k_na_fill(const double *__restrict__ x, int n, int nbx, int nby, int *scratch,
                          const int *__restrict__ bin_start, int *bin_ids) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int b = bin_index(x[2 * p], x[2 * p + 1], nbx, nby);
        bin_ids[bin_start[b] + atomicAdd(&scratch[MAX_BINS + b], 1)] = p;
    }
}

// ascending ids within each bin (insertion sort by one thread per bin)
__global__ void k_na_sort(const int *__restrict__ bin_start, int *bin_ids, int nbins) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
        const int s = bin_start[b], e = bin_start[b + 1];
        for (int i = s + 1; i < e; ++i) {
            const int v = bin_ids[i];
            int j = i - 1;
            while (j >= s && bin_ids[j] > v) {
                bin_ids[j + 1] = bin_ids[j];
                --j;
            }
            bin_ids[j + 1] = v;
        }
    }
}

}  // namespace

extern "C" int imb_bin_particles_noalloc(const double *d_x, int n, int nx, int ny, int *d_bin_start,
                                         int *d_bin_ids, void *stream) {
    if (nx < 1 || ny < 1 || n < 0 || (n > 0 && (!d_x || !d_bin_ids)) || !d_bin_start)
        return IMB_E_INVALID_ARG;
    const int nbx = (nx + imb::TILE - 1) / imb::TILE, nby = (ny + imb::TILE - 1) / imb::TILE;
    if ((long long)nbx * nby > MAX_BINS) return IMB_E_INVALID_ARG;   // beyond the fixed scratch
    const int nbins = nbx * nby;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return IMB_E_CUDA;
    if (stream) {   // the scratch address below is the current device's
        int sdev = -1;
        if (cudaStreamGetDevice((cudaStream_t)stream, &sdev) != cudaSuccess) return IMB_E_CUDA;
        if (sdev != dev) return IMB_E_INVALID_ARG;
    }
    int *scratch;
    {
        // first call on this device: the host-side name of the array is not a device
        // address, so look the address up (with this device current) and keep it
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_ptr[dev]) {
            int *p = nullptr;
            if (cudaGetSymbolAddress((void **)&p, g_bin_scratch) != cudaSuccess || !p) return IMB_E_CUDA;
            g_scratch_ptr[dev] = p;
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int gb = (nbins + 255) / 256, gp = n > 0 ? (n + 255) / 256 : 1;
    k_na_clear<<<gb, 256, 0, s>>>(scratch, nbins);
    if (n > 0) k_na_count<<<gp, 256, 0, s>>>(d_x, n, nbx, nby, scratch);
    k_na_scan<<<1, 1024, 0, s>>>(scratch, d_bin_start, nbins);
    if (n > 0) {
        k_na_fill<<<gp, 256, 0, s>>>(d_x, n, nbx, nby, scratch, d_bin_start, d_bin_ids);
        k_na_sort<<<gb, 256, 0, s>>>(d_bin_start, d_bin_ids, nbins);
    }
    return cudaGetLastError() == cudaSuccess ? IMB_OK : IMB_E_CUDA;
}
