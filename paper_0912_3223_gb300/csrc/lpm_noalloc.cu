// lpm_noalloc.cu - lpm_draws_static: the draws of lpm_draws without any device allocation.
//
// lpm_draws stages its inputs and outputs in device buffers it allocates on every call.
// Some callers cannot allow that: an application whose device memory is owned by its own
// pool allocator or capped by a fixed budget, or a host thread that must not take the
// driver's allocation path while other work is in flight. This variant stages through
// one file-scope device array of fixed size instead, so it calls no cudaMalloc,
// cudaFree or allocating library routine.
#include <cstdio>
#include <mutex>

#include "../../include/lpm.h"
#include "lpm_launch.h"

namespace {

constexpr long long kMax = LPM_DRAWS_STATIC_MAX;
constexpr int kMaxDevices = 64;
// layout of the scratch: pid [kMax] u64 | step [kMax] u32 | words [kMax] 4 x u32 |
// normals [kMax] 3 x f32
constexpr size_t kPidOff = 0;
constexpr size_t kStepOff = kPidOff + sizeof(unsigned long long) * kMax;
constexpr size_t kWordsOff = kStepOff + sizeof(unsigned int) * kMax;
constexpr size_t kNrmOff = kWordsOff + sizeof(uint4) * kMax;
constexpr size_t kBytes = kNrmOff + sizeof(float) * 3 * kMax;
static_assert(kWordsOff % 16 == 0, "uint4 staging must be 16-byte aligned");

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_draws_scratch[kBytes];

std::mutex g_mutex;
void *g_scratch[kMaxDevices] = {};   // device address of g_draws_scratch per device

lpm_status fail(lpm_status s, const char *msg)
{
    lpm::set_global_error(msg);
    return s;
}

lpm_status fail_cuda(const char *what, cudaError_t e)
{
    (void)cudaGetLastError();    // reported through the status; do not let it linger
    char buf[256];
    std::snprintf(buf, sizeof buf, "lpm_draws_static: %s: %s", what, cudaGetErrorString(e));
    return fail(e == cudaErrorMemoryAllocation ? LPM_E_OOM : LPM_E_CUDA, buf);
}

}  // namespace

extern "C" lpm_status lpm_draws_static(uint64_t seed, const uint64_t *pid, const uint32_t *step,
                                       uint32_t stream, int64_t n, uint32_t *words, float *normals)
{
    lpm::set_global_error("");
    if (n < 0 || (n > 0 && (!pid || !step || !words || !normals)))
        return fail(LPM_E_INVALID, "lpm_draws_static: invalid arguments");
    if (n > kMax) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "lpm_draws_static: n = %lld exceeds the %lld draws of the "
                      "static scratch (use lpm_draws)", (long long)n, kMax);
        return fail(LPM_E_INVALID, buf);
    }
    if (n == 0) return LPM_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda("cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return fail(LPM_E_INVALID, "lpm_draws_static: device ordinal too large");
    unsigned char *base;
    {
        // set-up, once per device, with that device current: the host-side name of the
        // array is not a device address, so look the address up
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_draws_scratch);
            if (e != cudaSuccess || !p) return fail_cuda("cudaGetSymbolAddress", e);
            g_scratch[dev] = p;
        }
        base = static_cast<unsigned char *>(g_scratch[dev]);
    }
    auto *d_pid = reinterpret_cast<unsigned long long *>(base + kPidOff);
    auto *d_step = reinterpret_cast<unsigned int *>(base + kStepOff);
    auto *d_words = reinterpret_cast<uint4 *>(base + kWordsOff);
    auto *d_nrm = reinterpret_cast<float *>(base + kNrmOff);
    e = cudaMemcpy(d_pid, pid, n * sizeof(unsigned long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_step, step, n * sizeof(unsigned int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail_cuda("copying the inputs", e);
    e = lpm::launch_draws(nullptr, seed, d_pid, d_step, stream, n, d_words, d_nrm);
    if (e != cudaSuccess) return fail_cuda("launch", e);
    e = cudaMemcpy(words, d_words, n * sizeof(uint4), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(normals, d_nrm, n * 3 * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda("copying the outputs", e);
    return LPM_OK;
}
