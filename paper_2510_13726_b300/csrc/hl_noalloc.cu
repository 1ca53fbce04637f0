// Total mass of a population array without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// mass total: code running inside a memory pool that forbids new
// allocations, a host driver that has handed all device memory to the
// lattice, or a callback whose allocator is not re-entrant.  This entry point
// keeps its block partials in a fixed array in the library's own static
// device memory, so the caller passes only the populations and the output.
//
// The array holds MAX_CHUNKS partial sums, one per chunk of 2^20 stored
// values, so at most MAX_CHUNKS * 2^20 = 2^32 values (q * n_cells) are
// accepted.  Every GPU that loads the library holds the array until the
// process exits.
#include <mutex>

#include "hl_internal.h"
#include "hlbm.h"

namespace {

constexpr int NA_MAX_CHUNKS = 4096;
constexpr long long NA_CHUNK = 1LL << 20;
constexpr int NA_THREADS = 256;
constexpr int NA_MAX_DEVICES = 64;

struct NoAllocScratch {
    double partial[NA_MAX_CHUNKS];
    unsigned done;
};

static __device__ __align__(256) NoAllocScratch na_scratch;

std::mutex na_mutex;
NoAllocScratch* na_ptr[NA_MAX_DEVICES] = {nullptr};

template <int S>
__global__ void __launch_bounds__(NA_THREADS) mass_noalloc_kernel(const void* fv, long long count, double shift,
                                                                  NoAllocScratch* sc, double* out) {
    using T = typename hl::Store<S>::T;
    const T* f = static_cast<const T*>(fv);
    const long long lo = (long long)blockIdx.x * NA_CHUNK;
    const long long hi = lo + NA_CHUNK < count ? lo + NA_CHUNK : count;
    double v = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += NA_THREADS) v += (double)hl::Store<S>::ld(f + i);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __shared__ double sh[NA_THREADS / 32];
    __shared__ bool last;
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) s += sh[w];
        sc->partial[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(&sc->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += ((volatile double*)sc->partial)[b];
        *out = s + shift;
        sc->done = 0u;
    }
}

// Address of the static scratch on the current device, looked up once per
// device (cudaGetSymbolAddress needs that device current).
cudaError_t scratch_for_current_device(NoAllocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(na_mutex);
    if (!na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, na_scratch);
        if (e != cudaSuccess) return e;
        na_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = na_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" hl_status hl_mass_noalloc(int q, int storage, const void* d_f, long long n_cells, double* d_mass,
                                     void* stream) {
    if ((q != 19 && q != 27) || storage < 0 || storage > 2 || !d_f || !d_mass || n_cells <= 0)
        return HL_ERR_ARG;
    const long long count = (long long)q * n_cells;
    const long long chunks = (count + NA_CHUNK - 1) / NA_CHUNK;
    if (chunks > NA_MAX_CHUNKS) return HL_ERR_WORKSPACE;   // more than 2^32 stored values
    // an error left pending by earlier, unrelated work belongs to that work:
    // report it (and clear it, as any runtime call would) before launching,
    // so that the launch check below sees this call's launch only
    if (cudaGetLastError() != cudaSuccess) return HL_ERR_CUDA;
    NoAllocScratch* sc = nullptr;
    if (scratch_for_current_device(&sc) != cudaSuccess) return HL_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the completion counter must start at zero even if an earlier call was cut short
    if (cudaMemsetAsync(&sc->done, 0, sizeof(unsigned), s) != cudaSuccess) return HL_ERR_CUDA;
    // storage shift: the stored values are f_i - w_i; sum_i w_i = 1 on D3Q19 and D3Q27
    const double shift = (double)n_cells;
    switch (storage) {
        case HL_STORE_F32: mass_noalloc_kernel<hl::ST_F32><<<(unsigned)chunks, NA_THREADS, 0, s>>>(d_f, count, shift, sc, d_mass); break;
        case HL_STORE_F16S: mass_noalloc_kernel<hl::ST_F16S><<<(unsigned)chunks, NA_THREADS, 0, s>>>(d_f, count, shift, sc, d_mass); break;
        default: mass_noalloc_kernel<hl::ST_BF16S><<<(unsigned)chunks, NA_THREADS, 0, s>>>(d_f, count, shift, sc, d_mass); break;
    }
    return cudaGetLastError() == cudaSuccess ? HL_OK : HL_ERR_CUDA;
}
