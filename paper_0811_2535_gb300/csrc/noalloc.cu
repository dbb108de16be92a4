// moa_fft_exec_noalloc: a 1-D transform that allocates no memory.
//
// Some callers cannot call cudaMalloc at all: code running where the CUDA
// allocator is off limits (a custom allocator owns all device memory, a
// real-time path that must never block in the driver, a plugin whose host
// forbids allocation after start-up).  For them this entry point runs the
// same kernels as moa_fft_exec on a single 1-D transform of n <= 2^20
// points, with its scratch (the r x c intermediate of the lifted transform)
// and its twiddle tables in file-scope static device arrays.  These arrays
// exist once per device in every process that loads the library and live
// until the process exits.
//
// Set-up happens on the first call on each device: the device addresses of
// the arrays are looked up with cudaGetSymbolAddress (in host code the array
// names are only host-side stand-ins, not device addresses), the twiddle
// tables are generated and the caller's stream is synchronised once.  Make
// that first call before any stream capture.
//
// All calls on one device share the arrays, which keep the last call's
// contents (nothing in them needs to start at zero except the status word).
// Calls on one device that overlap on the GPU, for instance on two streams,
// race on the scratch and the status word; calls on different devices do not
// interact.
//
// The status word collects what the kernels' bounded waits report
// (MOA_ERR_TIMEOUT); moa_fft_noalloc_status reads it after the caller's work
// on a stream and clears it.  A call does not clear it, so an error stays
// until it is read.
//
// If the device's context is destroyed and made again (cudaDeviceReset),
// the module is loaded afresh: the arrays get new addresses and lose their
// tables.  Every call therefore looks the scratch array's address up again
// (a host-side lookup) and repeats the set-up when it has moved.
#include <cuda_runtime.h>

#include <cstdlib>
#include <mutex>

#include "fft_core.cuh"
#include "internal.h"
#include "moa_fft.h"

namespace {

constexpr int kMaxLogN = 20;                       // largest transform: 2^20 points
constexpr int64_t kScratchElems = int64_t(1) << kMaxLogN;
constexpr int kStageEntries = 8192;                // all stage tables, N = 2..4096 (6912 used)
constexpr int kLiftHalf = 1 << ((kMaxLogN + 1) / 2);   // entries of each two-level half

// Scratch: the lifted transform's intermediate B' (n complex64 values, 8 MiB).
static __device__ __align__(256) float2 g_scratch[kScratchElems];
// Stage twiddle tables for every N = 2^1..2^12, back to back.
static __device__ __align__(256) float2 g_stage_tw[kStageEntries];
// Two-level tables w_n^e for n = 2^13..2^20: [log n - 13][lo | hi][kLiftHalf].
static __device__ __align__(256) float2 g_lift_tw[kMaxLogN - 12][2][kLiftHalf];
// Status word for the kernels' bounded waits.
static __device__ __align__(256) int g_status;

struct DeviceState {
    bool ready = false;
    float2 *scratch = nullptr;
    float2 *stage = nullptr;
    float2 *lift = nullptr;
    int *status = nullptr;
    int stage_off[13] = {0};
};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
DeviceState g_dev[kMaxDevices];

int ilog2(int64_t v)
{
    int l = 0;
    while ((int64_t(1) << l) < v)
        ++l;
    return l;
}

moa_status_t setup(int dev, cudaStream_t stream, DeviceState &st)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess)
        return MOA_ERR_CUDA;
    st.scratch = static_cast<float2 *>(p);
    if (cudaGetSymbolAddress(&p, g_stage_tw) != cudaSuccess)
        return MOA_ERR_CUDA;
    st.stage = static_cast<float2 *>(p);
    if (cudaGetSymbolAddress(&p, g_lift_tw) != cudaSuccess)
        return MOA_ERR_CUDA;
    st.lift = static_cast<float2 *>(p);
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess)
        return MOA_ERR_CUDA;
    st.status = static_cast<int *>(p);
    (void)dev;

    if (moa::prepare_kernels() != cudaSuccess || moa::prepare_pipe_kernels() != cudaSuccess)
        return MOA_ERR_CUDA;
    int off = 0;
    for (int l = 1; l <= 12; ++l) {
        const int ent = moa::stage_table_entries(l);
        st.stage_off[l] = off;
        if (ent > 0) {
            if (off + ent > kStageEntries)
                return MOA_ERR_UNSUPPORTED;
            if (moa::generate_stage_table(st.stage + off, l, stream) != cudaSuccess)
                return MOA_ERR_CUDA;
            off += (ent + 31) & ~31;
        }
    }
    for (int logn = 13; logn <= kMaxLogN; ++logn) {
        float2 *lo = st.lift + (size_t)(logn - 13) * 2 * kLiftHalf;
        if (moa::generate_two_level(lo, lo + kLiftHalf, logn, (logn + 1) / 2, stream) != cudaSuccess)
            return MOA_ERR_CUDA;
    }
    if (cudaMemsetAsync(st.status, 0, sizeof(int), stream) != cudaSuccess)
        return MOA_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess)
        return MOA_ERR_CUDA;
    st.ready = true;
    return MOA_OK;
}

// The device's arrays, set up for the current context: the scratch array's
// address is looked up again and compared with the one the set-up recorded.
moa_status_t ready_state(int dev, cudaStream_t s, DeviceState &out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess)
        return MOA_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState &st = g_dev[dev];
    if (st.ready && st.scratch != static_cast<float2 *>(p))
        st.ready = false;   // the context was made again: the arrays moved
    if (!st.ready) {
        const moa_status_t rc = setup(dev, s, st);
        if (rc != MOA_OK)
            return rc;
    }
    out = st;
    return MOA_OK;
}

}  // namespace

extern "C" moa_status_t moa_fft_exec_noalloc(const void *in, void *out, int64_t n, int sign, void *stream)
{
    if (!in || !out || (sign != 1 && sign != -1))
        return MOA_ERR_INVALID_ARG;
    if (n < 2 || (n & (n - 1)) != 0)
        return MOA_ERR_INVALID_SIZE;
    if (n > kScratchElems)
        return MOA_ERR_UNSUPPORTED;   // beyond the static scratch (2^20 points)
    if ((reinterpret_cast<uintptr_t>(in) & 7) || (reinterpret_cast<uintptr_t>(out) & 7))
        return MOA_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return MOA_ERR_CUDA;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceState st;
    const moa_status_t rc = ready_state(dev, s, st);
    if (rc != MOA_OK)
        return rc;

    moa::TwiddleSet tw{};
    for (int l = 1; l <= 12; ++l)
        tw.stage[l] = moa::stage_table_entries(l) > 0 ? st.stage + st.stage_off[l] : nullptr;
    const int L = ilog2(n);
    // fault injection for tests (MOA_FAULT_WAIT=1 at call time): the
    // pipelined kernels give up on a tile load that has not landed at its
    // first test
    const char *fw = std::getenv("MOA_FAULT_WAIT");
    const int fault = (fw && std::atoi(fw) == 1) ? moa::FLAG_SHORT_WAIT : 0;
    const int first = (sign > 0 ? moa::FLAG_CONJ_IN : 0) | fault;
    const int last = (sign > 0 ? moa::FLAG_CONJ_OUT : 0) | fault;
    const bool pipe_ok = moa::pipe_supported();
    const float2 *src = static_cast<const float2 *>(in);
    float2 *dst = static_cast<float2 *>(out);
    if (L <= 12) {
        moa::PassDesc d{};
        d.kind = moa::PASS_ROW;
        d.logN = L;
        d.O = 1;
        d.C = 1;
        d.Rt = 1;
        d.logF = moa::pick_logF_row(L, 1, false);
        return moa::launch_pass(d, src, dst, tw, first | last, s, st.status) == cudaSuccess ? MOA_OK
                                                                                            : MOA_ERR_CUDA;
    }
    const int lr = L / 2, lc = L - lr;
    const int64_t r = int64_t(1) << lr, c = int64_t(1) << lc;
    float2 *lift = st.lift + (size_t)(L - 13) * 2 * kLiftHalf;
    tw.lo = lift;
    tw.hi = lift + kLiftHalf;
    tw.h = (L + 1) / 2;

    moa::PassDesc p1{};
    p1.kind = moa::PASS_COL;
    p1.logN = lr;
    p1.O = 1;
    p1.C = c;
    p1.Rt = 1;
    p1.logF = moa::pick_logF_col(lr, c);
    p1.tw4 = 1;
    p1.pipe = pipe_ok && lr >= 10 && p1.logF == 2 && c >= 4;
    moa::PassDesc p2{};
    p2.kind = moa::PASS_ROW;
    p2.logN = lc;
    p2.O = r;
    p2.C = 1;
    p2.Rt = r;
    p2.logF = moa::pick_logF_row(lc, r, true);
    p2.pipe = pipe_ok && lc >= 10 && p2.logF == 2;
    if (moa::launch_pass(p1, src, st.scratch, tw, first, s, st.status) != cudaSuccess)
        return MOA_ERR_CUDA;
    if (moa::launch_pass(p2, st.scratch, dst, tw, last, s, st.status) != cudaSuccess)
        return MOA_ERR_CUDA;
    return MOA_OK;
}

extern "C" moa_status_t moa_fft_noalloc_status(void *stream)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return MOA_ERR_CUDA;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceState st;
    const moa_status_t rc = ready_state(dev, s, st);
    if (rc != MOA_OK)
        return rc;
    int word = 0;
    if (cudaMemcpyAsync(&word, st.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemsetAsync(st.status, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return MOA_ERR_CUDA;
    return static_cast<moa_status_t>(word);
}
