// kmx_match_noalloc: exact FP32 mutual matching that allocates nothing.
//
// Some callers cannot allocate device memory when they match: a process whose
// memory pool has already claimed the device, a real-time loop that must not
// block on the driver's allocator, or a host framework that forbids
// allocation calls from plug-in code.  This entry point computes the result
// of kmx_match(..., KMX_MATCH_FP32_EXACT, ...) with the dense exact tile
// kernel of match_fp32.cu (register-prefetched tiles, every dimension visited)
// followed by the shared merge, scan and emission of match_common.cu, and
// takes its scratch from a fixed array in device memory that is reserved when
// the library's module is loaded on a device and stays reserved until the
// process exits.
#include <cuda.h>

#include <mutex>

#include "kmx_internal.cuh"
#include "match_common.cuh"

namespace {

constexpr int64_t kMaxRows = KMX_NOALLOC_MAX_ROWS;
constexpr size_t kErrBytes = 256;                 // device error word, own 256-byte slot
constexpr size_t kStatusBytes = 256;              // the scan's look-back words (32 words)
constexpr size_t kScratchBytes = 6u << 20;        // >= error slot + match scratch for kMaxRows x kMaxRows

// The scratch.  In host code this name is only a stand-in for the symbol:
// kernels get the device address obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
// Device address of g_scratch per device, with the CUDA context it was looked
// up in: the address belongs to that context's copy of the module, so a call
// made under another context (after cudaDeviceReset, or with a non-primary
// context current) looks it up again.
struct Cached {
    CUcontext ctx;
    void* addr;
};
Cached g_addr[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn g_ctx_get_current = nullptr;

// The current CUDA context, through the driver entry point the runtime hands
// out (the library does not link the driver library itself).
kmx_status current_context(CUcontext* out)
{
    if (!g_ctx_get_current) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return KMX_ECUDA;
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    }
    CUcontext c = nullptr;
    if (g_ctx_get_current(&c) != CUDA_SUCCESS || !c) return KMX_ECUDA;
    *out = c;
    return KMX_OK;
}

// With the device current: the array's address in the current context,
// looked up once per device and context.
kmx_status scratch_address(int device, void** out)
{
    if (device < 0 || device >= kMaxDevices) return KMX_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    CUcontext ctx = nullptr;
    const kmx_status st = current_context(&ctx);
    if (st != KMX_OK) return st;
    if (!g_addr[device].addr || g_addr[device].ctx != ctx) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return KMX_ECUDA;
        g_addr[device].ctx = ctx;
        g_addr[device].addr = p;
    }
    *out = g_addr[device].addr;
    return KMX_OK;
}

// Last step of every call: a look-back wait of the scan that ran out leaves
// wrong offsets behind, and the error word that records it sits in the fixed
// array where no caller can read it; report it through the count instead.
__global__ void report_timeout(const unsigned int* __restrict__ err, int64_t* __restrict__ n_out)
{
    if (threadIdx.x == 0 && (*err & KMX_DERR_TIMEOUT)) *n_out = -1;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" kmx_status kmx_match_noalloc(const float* d_desc_p, const int32_t* d_valid_p, int64_t np_cap,
                                        const int64_t* d_np, const float* d_desc_q, const int32_t* d_valid_q,
                                        int64_t nq_cap, const int64_t* d_nq, kmx_corr* d_out, int64_t cap,
                                        int64_t* d_n_out, void* cuda_stream)
{
    if (np_cap < 0 || nq_cap < 0 || np_cap > kMaxRows || nq_cap > kMaxRows || cap < 0 || !d_n_out ||
        (np_cap > 0 && (!d_desc_p || !aligned16(d_desc_p))) || (nq_cap > 0 && (!d_desc_q || !aligned16(d_desc_q))) ||
        (cap > 0 && !d_out))
        return KMX_EINVAL;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) return KMX_ECUDA;
    void* base = nullptr;
    kmx_status st = scratch_address(device, &base);
    if (st != KMX_OK) return st;
    kmx_ctx c{};  // a stack context: no allocation, scratch and error word point into g_scratch
    c.device = device;
    c.stream = static_cast<cudaStream_t>(cuda_stream);
    c.d_err = static_cast<unsigned int*>(base);
    // the scan's status words sit in the array too, so it never grows them
    c.scan_status = reinterpret_cast<unsigned long long*>(static_cast<char*>(base) + kErrBytes);
    c.scan_words = kStatusBytes / sizeof(unsigned long long);
    c.ws = static_cast<char*>(base) + kErrBytes + kStatusBytes;
    c.ws_size = kScratchBytes - kErrBytes - kStatusBytes;
    if (kmx_scan_words(np_cap) > c.scan_words) return KMX_EINVAL;  // cannot happen for np_cap <= kMaxRows
    if (cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return KMX_ECUDA;
    if (np_cap == 0 || nq_cap == 0)
        return cudaMemsetAsync(d_n_out, 0, sizeof(int64_t), c.stream) == cudaSuccess ? KMX_OK : KMX_ECUDA;
    int chunks = 0;
    const size_t need = kmx_match_fp32_scratch_bytes(np_cap, nq_cap, &chunks);
    if (need > c.ws_size) return KMX_EINVAL;
    kmx::MatchScratch s = kmx::match_common_carve(c.ws, np_cap, nq_cap, chunks);
    // the array keeps the previous call's contents: reset what must start fresh
    cudaError_t e = cudaMemsetAsync(c.d_err, 0, sizeof(unsigned int), c.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.scan_status, 0, kStatusBytes, c.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.colbest, 0xFF, sizeof(unsigned long long) * nq_cap, c.stream);
    if (e == cudaSuccess) e = kmx_match_fp32_launch(&c, d_desc_p, np_cap, d_np, d_desc_q, nq_cap, d_nq, s, chunks);
    if (e == cudaSuccess) e = kmx::match_finalize(&c, s, np_cap, d_np, d_valid_p, d_valid_q, d_out, cap, d_n_out);
    if (e == cudaSuccess) {
        KMX_COUNT_LAUNCH();
        report_timeout<<<1, 32, 0, c.stream>>>(c.d_err, d_n_out);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? KMX_OK : KMX_ECUDA;
}
