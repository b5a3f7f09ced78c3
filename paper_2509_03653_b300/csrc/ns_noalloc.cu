// ns_noalloc.cu -- ns_window_stats_static: the nine statistics of one small
// window with every working table in a fixed device array, so the call
// itself never allocates device memory.
//
// Who needs this: callers that cannot call cudaMalloc at the point they need
// the statistics -- a process whose device memory is already fully claimed by
// another framework's caching allocator, or a latency-critical capture loop
// that must never block in cudaMalloc / cudaFree (both may synchronize the
// whole device).  They still pass their own input columns and output record.
//
// The array below is a file-scope __device__ object: every GPU that loads
// the library holds it (kScratchBytes, about 3 MiB) until the process exits.
// Host code must not pass its name to a kernel (on the host the name is only
// a stand-in, not a device address); the first call on each device looks up
// the real address with cudaGetSymbolAddress, with that device current, and
// caches it.
#include <cstdio>
#include <mutex>

#include "ns.h"
#include "ns_api_internal.h"
#include "ns_common.cuh"
#include "ns_kernels.h"

namespace {

using namespace ns;

constexpr u64 kMaxPackets = NS_STATIC_MAX_PACKETS;
constexpr u64 kCap = 2 * kMaxPackets;  // link/row/column slots: load <= 1/2
static_assert((kCap & (kCap - 1)) == 0, "capacity must be a power of two");

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kLinksOff = 0;
constexpr size_t kRowsOff = align256(kLinksOff + (kCap + 1) * sizeof(LinkSlot));
constexpr size_t kColsOff = align256(kRowsOff + (kCap + 1) * sizeof(NodeSlot));
constexpr size_t kStatsOff = align256(kColsOff + (kCap + 1) * sizeof(NodeSlot));
constexpr size_t kScratchBytes = align256(kStatsOff + sizeof(DevStats));

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

struct DeviceSetup {
    bool ready = false;
    unsigned char* base = nullptr;  // device address of g_static_scratch
    int sms = 0;
};

constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

thread_local char g_msg[256];

}  // namespace

extern "C" ns_status ns_window_stats_static(const uint32_t* d_src, const uint32_t* d_dst, uint64_t n,
                                            ns_stats* d_out, ns_stream_t stream) {
    if (!d_out) return ns::set_fail(NS_ERR_INVALID, "ns_window_stats_static: d_out is NULL");
    if (n > 0 && (!d_src || !d_dst))
        return ns::set_fail(NS_ERR_INVALID, "ns_window_stats_static: NULL input with n > 0");
    if (n > kMaxPackets) {
        snprintf(g_msg, sizeof g_msg,
                 "ns_window_stats_static: n = %llu exceeds the fixed maximum of %llu packets per call",
                 (unsigned long long)n, (unsigned long long)kMaxPackets);
        return ns::set_fail(NS_ERR_INVALID, g_msg);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return ns::set_fail(NS_ERR_CUDA, "ns_window_stats_static: no usable current device");
    }
    DeviceSetup su;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_setup[dev].ready) {
            // once per device, with that device current
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || p == nullptr) {
                snprintf(g_msg, sizeof g_msg, "ns_window_stats_static: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
                cudaGetLastError();
                return ns::set_fail(NS_ERR_CUDA, g_msg);
            }
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
                sms = 1;
            g_setup[dev].base = (unsigned char*)p;
            g_setup[dev].sms = sms;
            g_setup[dev].ready = true;
        }
        su = g_setup[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the array looked up above is the current device's: a stream of another
    // device could not reach it
    int sdev = dev;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) {
        cudaGetLastError();
        return ns::set_fail(NS_ERR_INVALID, "ns_window_stats_static: not a valid stream");
    }
    if (sdev != dev) {
        snprintf(g_msg, sizeof g_msg,
                 "ns_window_stats_static: the stream belongs to device %d, the current device is %d", sdev, dev);
        return ns::set_fail(NS_ERR_INVALID, g_msg);
    }
    // every call shares the array: start from empty tables and zero statistics
    cudaError_t e = cudaMemsetAsync(su.base, 0, kScratchBytes, s);
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof g_msg, "ns_window_stats_static: clearing the tables failed: %s",
                 cudaGetErrorString(e));
        return ns::set_fail(NS_ERR_CUDA, g_msg);
    }
    HashView v;
    v.links = (LinkSlot*)(su.base + kLinksOff);
    v.link_mask = kCap - 1;
    v.rows = (NodeSlot*)(su.base + kRowsOff);
    v.row_mask = kCap - 1;
    v.cols = (NodeSlot*)(su.base + kColsOff);
    v.col_mask = kCap - 1;
    v.stats = (DevStats*)(su.base + kStatsOff);
    launch_insert_packets(d_src, d_dst, n, v, su.sms, true, s);
    launch_stats_out(v.stats, (u64*)d_out, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof g_msg, "ns_window_stats_static: launch failed: %s", cudaGetErrorString(e));
        return ns::set_fail(NS_ERR_CUDA, g_msg);
    }
    return NS_OK;
}
