// Allocation-free variant of igamg_extrapolate.
//
// Some callers cannot allocate device memory at the point where they need an
// extrapolation step: code embedded in a host framework that owns every device
// allocation and forbids cudaMalloc on its hot path (cudaMalloc can block the
// whole device and can fail when memory is fragmented), or code running under
// a fixed memory budget with no allocator handle to pass scratch through.
// This entry point takes its scratch from a fixed array compiled into the
// library instead of from a caller-provided workspace.  The caller still
// passes the iterates (input) and the extrapolant (output).
//
// The array lives in device memory of every GPU that loads the library, for
// the lifetime of the process.  All calls share it and it keeps whatever the
// last call left there; the kernels write every scratch word before reading
// it, so nothing needs clearing between calls.  Calls whose GPU work overlaps
// (for example on two streams) race on the array and give wrong results:
// serialise them.
#include "../../include/igamg.h"
#include "device.hpp"

#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

namespace {

// 240 KiB: the Gram partials for the largest restart number (304 blocks x 91
// entries x 8 bytes = 221,312 bytes) plus the coefficients, the used-q word
// and the pass-1 state of the CholeskyQR2 extrapolation.
constexpr size_t kScratchBytes = 240 * 1024;
static __device__ __align__(256) unsigned char g_extrap_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};     // device address of the array, per device

igamg_status fail(igamg_status st, const std::string& msg) {
    igamg::set_last_error(msg);        // reported by igamg_last_error()
    return st;
}

// Device address of the scratch array on the current device.  The array's
// name in host code is only a host-side stand-in, so the address is looked up
// once per device with cudaGetSymbolAddress (with that device current).
igamg_status scratch_for_current_device(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(IGAMG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(IGAMG_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_extrap_scratch);
        if (e != cudaSuccess || !p)
            return fail(IGAMG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return IGAMG_OK;
}

}  // namespace

extern "C" {

igamg_status igamg_extrapolate_noalloc(long n, int q, int method, const double* d_S, long ld, double* d_t,
                                       double* h_gamma, int* h_qused, void* stream) {
    if (n <= 0 || q < 1 || q > igamg::kMaxQ || (method != IGAMG_RRE && method != IGAMG_MPE) || !d_S || !d_t ||
        ld < n)
        return fail(IGAMG_EINVAL, "bad extrapolation arguments");
    const int nb = igamg::dev::gram_blocks((size_t)n);
    const size_t np = (size_t)(q + 1) * (q + 2) / 2;
    const size_t part_bytes = ((size_t)nb * np * 8 + 255) / 256 * 256;
    const size_t need = part_bytes + 512 + (sizeof(igamg::ExtrapInfo) + 255) / 256 * 256;
    if (need > kScratchBytes)
        return fail(IGAMG_EINVAL, "scratch needed (" + std::to_string(need) + " bytes) exceeds the built-in " +
                                      std::to_string(kScratchBytes) + " bytes");
    void* base = nullptr;
    if (igamg_status st = scratch_for_current_device(&base)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double* partial = (double*)base;
    char* tail = (char*)base + part_bytes;
    double* gamma = (double*)tail;
    int* qused = (int*)(tail + 256);
    igamg::ExtrapInfo* info = (igamg::ExtrapInfo*)(tail + 512);
    igamg::dev::extrap_gammas(s, q, method, d_S, (size_t)ld, (size_t)n, partial, nb, info, gamma, qused);
    igamg::dev::combine(s, q, gamma, d_S, (size_t)ld, (size_t)n, d_t);
    double hg[igamg::kMaxQ + 2];
    int hq = 0;
    cudaError_t e = cudaMemcpyAsync(hg, gamma, (q + 2) * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hq, qused, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(IGAMG_ECUDA, std::string("extrapolation: ") + cudaGetErrorString(e));
    if (h_gamma) std::memcpy(h_gamma, hg, (q + 2) * sizeof(double));
    if (h_qused) *h_qused = hq;
    return IGAMG_OK;
}

}  // extern "C"
