// tf_stats.cu -- field statistics for the watchdog: sum of squares, largest
// magnitude and count of non-finite values of one stored field array.
//
// Two passes: one CTA per z plane reduces its plane to a partial (FP64 sum of
// squares, FP32 max |v|, 64-bit non-finite count) in scratch memory; one CTA
// reduces the partials.  Values are scaled to SI units on the way.
#include <math.h>

#include "tf_internal.cuh"

namespace tf {

namespace {
constexpr int kStatThreads = 256;

__device__ void block_reduce(double& s, float& m, unsigned long long& nf) {
    __shared__ double ss[kStatThreads / 32];
    __shared__ float sm[kStatThreads / 32];
    __shared__ unsigned long long sn[kStatThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
        nf += __shfl_down_sync(0xffffffffu, nf, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        ss[w] = s;
        sm[w] = m;
        sn[w] = nf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kStatThreads / 32; ++i) {
            s += ss[i];
            m = fmaxf(m, sm[i]);
            nf += sn[i];
        }
    }
}
}  // namespace

// pass 1: blockIdx.x = plane k of an (n0, n1, n2) array with row pitch `pitch`
__global__ void __launch_bounds__(kStatThreads) k_stats_planes(const float* f, int n0, int n1, int pitch,
                                                               long long plane, double scale, StatPartial* part) {
    const int k = blockIdx.x;
    const float* p = f + (long long)k * plane;
    double s = 0.0;
    float m = 0.f;
    unsigned long long nf = 0;
    const int npts = n0 * n1;
    for (int t = threadIdx.x; t < npts; t += kStatThreads) {
        // 64-bit offset: a caller's row pitch may make pitch * n1 exceed 2^31
        const float v = p[(long long)(t / n0) * pitch + (t % n0)];
        if (!isfinite(v)) {
            ++nf;
        } else {
            s += (double)v * (double)v;
            m = fmaxf(m, fabsf(v));
        }
    }
    block_reduce(s, m, nf);
    if (threadIdx.x == 0) {
        part[k].sumsq = s * scale * scale;
        part[k].maxabs = (double)m * fabs(scale);
        part[k].nonfinite = nf;
    }
}

// pass 2: one CTA reduces n partials into out
__global__ void __launch_bounds__(kStatThreads) k_stats_final(const StatPartial* part, int n, StatPartial* out) {
    __shared__ double ssum[kStatThreads], smax[kStatThreads];
    __shared__ unsigned long long snf[kStatThreads];
    double s = 0.0, mx = 0.0;
    unsigned long long nf = 0;
    for (int t = threadIdx.x; t < n; t += kStatThreads) {
        s += part[t].sumsq;
        mx = fmax(mx, part[t].maxabs);
        nf += part[t].nonfinite;
    }
    ssum[threadIdx.x] = s;
    smax[threadIdx.x] = mx;
    snf[threadIdx.x] = nf;
    __syncthreads();
    for (int o = kStatThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ssum[threadIdx.x] += ssum[threadIdx.x + o];
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
            snf[threadIdx.x] += snf[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out->sumsq = ssum[0];
        out->maxabs = smax[0];
        out->nonfinite = snf[0];
    }
}

cudaError_t launch_field_stats(const float* f, int n0, int n1, int n2, int pitch, long long plane, double scale,
                               StatPartial* partials, StatPartial* out, cudaStream_t st) {
    if (n2 < 1) return cudaErrorInvalidValue;
    k_stats_planes<<<n2, kStatThreads, 0, st>>>(f, n0, n1, pitch, plane, scale, partials);
    k_stats_final<<<1, kStatThreads, 0, st>>>(partials, n2, out);
    return cudaGetLastError();
}

}  // namespace tf

// ---------------------------------------------------------------------------
// Allocation-free variant.
//
// Some callers cannot allocate device memory at the moment they want the
// statistics: a monitoring thread that checks a running simulation for
// blow-ups must not take the CUDA allocator's lock or trigger the device-wide
// synchronisation that cudaFree implies, and a host application whose memory
// pool has already reserved (nearly) all of the device cannot get more.  For
// them the per-plane partials live in a fixed array of this file, sized for
// kNoAllocMaxPlanes planes, which every GPU that loads the library holds
// until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int kNoAllocMaxPlanes = 4096;
constexpr int kMaxDevices = 64;

// partials of one call followed by its result; shared by every call on a device
static __device__ __align__(256) tf::StatPartial g_stats_scratch[kNoAllocMaxPlanes + 1];

tf::StatPartial* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// device address of g_stats_scratch on the current device (looked up once per device)
cudaError_t scratch_address(tf::StatPartial** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_stats_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = (tf::StatPartial*)p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" tf_status tf_field_stats_noalloc(const float* field, int nx_pts, int ny_pts, int nz_pts, int pitch,
                                            double scale, double* sumsq, double* maxabs, int64_t* nonfinite,
                                            void* stream) {
    if (!field || nx_pts < 1 || ny_pts < 1 || nz_pts < 1 || pitch < nx_pts) return TF_EINVAL;
    if ((long long)nx_pts * ny_pts >= (1LL << 31)) return TF_EINVAL;
    if (nz_pts > kNoAllocMaxPlanes) return TF_EINVAL;   // beyond the fixed scratch
    tf::StatPartial* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return TF_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const long long plane = (long long)pitch * ny_pts;
    if (tf::launch_field_stats(field, nx_pts, ny_pts, nz_pts, pitch, plane, scale, scratch,
                               scratch + kNoAllocMaxPlanes, st) != cudaSuccess)
        return TF_ECUDA;
    tf::StatPartial r;
    if (cudaMemcpyAsync(&r, scratch + kNoAllocMaxPlanes, sizeof(r), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return TF_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return TF_ECUDA;
    if (sumsq) *sumsq = r.sumsq;
    if (maxabs) *maxabs = r.maxabs;
    if (nonfinite) *nonfinite = (int64_t)r.nonfinite;
    return TF_OK;
}
