// Morton order of a particle set on scratch that is part of the library image: the one entry
// point of the library that allocates no device memory at all.
//
// Some callers cannot let a library allocate while they run: an application that has already
// handed the device's free memory to its own pool (where cudaMalloc would fail), or one whose
// loop cannot take the device-wide synchronisation that cudaFree implies.  For them this file
// keeps a fixed scratch area in a file-scope __device__ array, sized for at most
// FMM_STATIC_ORDER_MAX_N particles, and fmm_morton_order_static sorts into the caller's buffers
// with it.  The device address of the array is looked up once per device, at the first call.
//
// The computation is the key and sort stage of fmm_build_tree (Sec. 3.1, hierarchically sorted
// order): same key arithmetic, same stable radix sort kernels, so the result is bit-identical.
#include <stdio.h>

#include <mutex>

#include "fmm_internal.cuh"
#include "morton.cuh"

fmm_status fmm_report_error(fmm_status st, const char* msg);

namespace {

constexpr long long kMaxN = FMM_STATIC_ORDER_MAX_N;
// scratch regions, each starting on a 256-byte boundary
constexpr long long kHistCap = 256LL * (kMaxN / 1024);  // digit counts: 256 per tile of >= 1024 keys
constexpr long long kPartCap = 4096;                     // partial sums of their scan
constexpr long long kOffKeyAlt = 0;
constexpr long long kOffIdxAlt = kOffKeyAlt + 8 * kMaxN;
constexpr long long kOffHist = kOffIdxAlt + 4 * kMaxN;
constexpr long long kOffPart = kOffHist + 4 * kHistCap;
constexpr long long kOffStatus = kOffPart + 4 * kPartCap;
constexpr long long kScratchBytes = kOffStatus + 256;  // 13,648,128 bytes
static_assert(kOffIdxAlt % 256 == 0 && kOffHist % 256 == 0 && kOffPart % 256 == 0 && kOffStatus % 256 == 0,
              "scratch regions must stay 256-byte aligned");

constexpr int kMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_order_scratch[kScratchBytes];

static std::mutex g_setup_mutex;
static unsigned char* g_scratch_ptr[kMaxDevices];  // device address of g_order_scratch, per device

static fmm_status report(fmm_status st, const char* fmt, long long a = 0, long long b = 0)
{
    char buf[256];
    snprintf(buf, sizeof buf, fmt, a, b);
    return fmm_report_error(st, buf);
}

static fmm_status report_cuda(cudaError_t e, const char* what)
{
    char buf[256];
    snprintf(buf, sizeof buf, "fmm_morton_order_static: %s: %s", what, cudaGetErrorString(e));
    return fmm_report_error(FMM_ERR_CUDA, buf);
}

// Once per device, with that device current: the array's device address and the sort's
// shared-memory attribute.  Later calls only read the table.
static fmm_status scratch_for(int dev, unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        if (fmm_sort_hist_entries(kMaxN) > kHistCap || fmm_sort_part_entries(kMaxN) > kPartCap)
            return report(FMM_ERR_STATE, "fmm_morton_order_static: internal scratch layout too small");
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_order_scratch);
        if (e != cudaSuccess) return report_cuda(e, "cudaGetSymbolAddress");
        if (!p) return report(FMM_ERR_CUDA, "fmm_morton_order_static: no device address for the scratch");
        e = fmm_sort_prepare();
        if (e != cudaSuccess) return report_cuda(e, "sort set-up");
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return FMM_OK;
}

// Morton key and identity index per particle; flags positions outside [0, 1)^3.
__global__ void k_order_keys(const double* __restrict__ pos, long long n, unsigned long long* __restrict__ key,
                             unsigned int* __restrict__ idx, unsigned int* __restrict__ status)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = pos[i], y = pos[n + i], z = pos[2 * n + i];
    if (!(x >= 0.0 && x < 1.0 && y >= 0.0 && y < 1.0 && z >= 0.0 && z < 1.0)) atomicOr(status, FMM_DEV_ERR_ARG);
    key[i] = (spread3(quantise21(x)) << 2) | (spread3(quantise21(y)) << 1) | spread3(quantise21(z));
    idx[i] = (unsigned int)i;
}

extern "C" fmm_status fmm_morton_order_static(const double* pos, long long n, unsigned long long* keys,
                                              unsigned int* order, void* cuda_stream)
{
    if (!pos || !keys || !order) return report(FMM_ERR_ARG, "fmm_morton_order_static: NULL argument");
    if (n < 1 || n > kMaxN)
        return report(FMM_ERR_ARG, "fmm_morton_order_static: n = %lld is outside [1, %lld], the size of its fixed scratch",
                      n, kMaxN);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return report(FMM_ERR_ARG, "fmm_morton_order_static: device %lld not supported", dev);
    unsigned char* base = nullptr;
    fmm_status st = scratch_for(dev, &base);
    if (st != FMM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned long long* key_alt = reinterpret_cast<unsigned long long*>(base + kOffKeyAlt);
    unsigned int* idx_alt = reinterpret_cast<unsigned int*>(base + kOffIdxAlt);
    unsigned int* hist = reinterpret_cast<unsigned int*>(base + kOffHist);
    unsigned int* part = reinterpret_cast<unsigned int*>(base + kOffPart);
    unsigned int* status = reinterpret_cast<unsigned int*>(base + kOffStatus);
    // the status word is the only scratch that must start at zero: the sort writes every digit
    // count and partial sum it reads
    e = cudaMemsetAsync(status, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return report_cuda(e, "clearing the status word");
    k_order_keys<<<(unsigned)fmm_ceil_div(n, 256), 256, 0, s>>>(pos, n, keys, order, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report_cuda(e, "key kernel");
    // 8 passes (an even number): the sorted keys and order end in the caller's buffers
    e = fmm_radix_sort_kv_scratch(keys, key_alt, order, idx_alt, n, 8, hist, part, s);
    if (e != cudaSuccess) return report_cuda(e, "radix sort");
    unsigned int st_h = 0;
    e = cudaMemcpyAsync(&st_h, status, sizeof st_h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return report_cuda(e, "reading the status word");
    if (st_h & FMM_DEV_ERR_ARG)
        return report(FMM_ERR_ARG, "fmm_morton_order_static: a position outside [0,1) (the order is not valid)");
    return FMM_OK;
}
