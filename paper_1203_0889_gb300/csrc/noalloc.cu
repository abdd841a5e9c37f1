// noalloc.cu -- an allocation-free variant of the near-field (P2P) kernel.
//
// fmm_direct_noalloc evaluates the direct sum over all particle pairs (the
// FMM with a single root leaf, where P2P is the whole computation) without
// allocating device memory.  It is meant for callers that cannot call
// cudaMalloc: a plug-in inside a host framework that owns all device memory
// and forbids allocations by its plug-ins, or a real-time loop that must
// neither wait on the allocator nor risk running out of memory once it has
// started.  The caller passes inputs and outputs; the kernel's scratch (the
// staged (x, y, z, q) records and the per-particle accumulators) lives in
// the file-scope array below, which every GPU that loads this library keeps
// until the process exits.
#include <algorithm>
#include <mutex>

#include "fmm_internal.cuh"

namespace {

// Largest system the allocation-free entry point accepts.
constexpr int64_t kNoAllocMaxN = 16384;
// Per particle: one staged record (x, y, z, q) and four accumulators
// (phi, d/dx, d/dy, d/dz), all FP64: 64 bytes, 1 MiB in total.
constexpr size_t kNoAllocScratchBytes = (size_t)kNoAllocMaxN * 8 * sizeof(double);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};
int g_noalloc_sms[kMaxDevices] = {};   // multiprocessors of each device, read with the address

constexpr int NA_THREADS = 128;
constexpr int NA_TILE = 512;

template <typename T>
__global__ void k_na_stage(int64_t n, const T* __restrict__ pos, const T* __restrict__ q, double4_32a* xq,
                           double* acc) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    xq[i] = make_double4_32a((double)pos[3 * i], (double)pos[3 * i + 1], (double)pos[3 * i + 2], (double)q[i]);
    acc[4 * i] = 0.0; acc[4 * i + 1] = 0.0; acc[4 * i + 2] = 0.0; acc[4 * i + 3] = 0.0;
}

// Block (b, s): targets [128 b, 128 b + 128), sources of slice s; partial sums
// are added into the accumulators.
__global__ void __launch_bounds__(NA_THREADS) k_na_p2p(int64_t n, int64_t slice, const double4_32a* __restrict__ xq,
                                                        double* acc) {
    __shared__ double4_32a buf[NA_TILE];
    int64_t i = blockIdx.x * (int64_t)NA_THREADS + threadIdx.x;
    int64_t j0 = blockIdx.y * slice, j1 = min(n, j0 + slice);
    double4_32a me = i < n ? xq[i] : make_double4_32a(0, 0, 0, 0);
    double phi = 0, gx = 0, gy = 0, gz = 0;
    for (int64_t jb = j0; jb < j1; jb += NA_TILE) {
        int take = (int)min((int64_t)NA_TILE, j1 - jb);
        __syncthreads();
        for (int k = threadIdx.x; k < take; k += NA_THREADS) buf[k] = xq[jb + k];
        __syncthreads();
        for (int k = 0; k < take; k++) {
            double4_32a s = buf[k];
            double dx = me.x - s.x, dy = me.y - s.y, dz = me.z - s.z;
            double r2 = dx * dx + dy * dy + dz * dz;
            double rinv = r2 > 0.0 ? rsqrt(r2) : 0.0;
            double qr = s.w * rinv;
            phi += qr;
            double qr3 = qr * rinv * rinv;
            gx -= qr3 * dx; gy -= qr3 * dy; gz -= qr3 * dz;
        }
    }
    if (i < n) {
        atomicAdd(&acc[4 * i], phi);
        atomicAdd(&acc[4 * i + 1], gx);
        atomicAdd(&acc[4 * i + 2], gy);
        atomicAdd(&acc[4 * i + 3], gz);
    }
}

template <typename T>
__global__ void k_na_finish(int64_t n, const double4_32a* __restrict__ xq, const double* __restrict__ acc,
                            T* phi, T* force, int field) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (phi) phi[i] = (T)acc[4 * i];
    if (force) {
        double s = field ? -1.0 : -xq[i].w;
        force[3 * i] = (T)(s * acc[4 * i + 1]);
        force[3 * i + 1] = (T)(s * acc[4 * i + 2]);
        force[3 * i + 2] = (T)(s * acc[4 * i + 3]);
    }
}

// Device address of the scratch array for the current device, looked up once
// per device (the symbol's host-side name is not a device address), and the
// device's multiprocessor count, read at the same time.
int scratch_for_current_device(void** out, int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { fmm_set_error("fmm_direct_noalloc: cudaGetDevice: %s", cudaGetErrorString(e)); return FMM_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) { fmm_set_error("fmm_direct_noalloc: device %d unsupported", dev); return FMM_ERR_ARG; }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            fmm_set_error("fmm_direct_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return FMM_ERR_CUDA;
        }
        int nsm = 0;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || nsm < 1) {
            fmm_set_error("fmm_direct_noalloc: cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
            return FMM_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
        g_noalloc_sms[dev] = nsm;
    }
    *out = g_noalloc_ptr[dev];
    *sms = g_noalloc_sms[dev];
    return FMM_OK;
}

template <typename T>
int direct_noalloc_typed(int64_t n, const T* pos, const T* q, T* phi, T* force, int field, cudaStream_t st,
                         void* scratch, int sms) {
    double4_32a* xq = (double4_32a*)scratch;
    double* acc = (double*)((char*)scratch + (size_t)kNoAllocMaxN * sizeof(double4_32a));
    unsigned nb = (unsigned)((n + NA_THREADS - 1) / NA_THREADS);
    k_na_stage<T><<<nb, NA_THREADS, 0, st>>>(n, pos, q, xq, acc);
    // spread the sources over enough slices to give every SM four blocks
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>(64, (4 * (int64_t)sms + nb - 1) / nb));
    int64_t slice = (n + splits - 1) / splits;
    splits = (n + slice - 1) / slice;
    k_na_p2p<<<dim3(nb, (unsigned)splits), NA_THREADS, 0, st>>>(n, slice, xq, acc);
    k_na_finish<T><<<nb, NA_THREADS, 0, st>>>(n, xq, acc, phi, force, field);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { fmm_set_error("fmm_direct_noalloc: %s", cudaGetErrorString(e)); return FMM_ERR_CUDA; }
    return FMM_OK;
}

}  // namespace

extern "C" int fmm_direct_noalloc(int64_t n, const void* pos, const void* q, void* phi, void* force, int dtype,
                                  int32_t flags, void* stream) {
    if (n < 0 || n > kNoAllocMaxN) {
        fmm_set_error("fmm_direct_noalloc: n=%lld outside [0, %lld] (the size of its static scratch)",
                      (long long)n, (long long)kNoAllocMaxN);
        return FMM_ERR_ARG;
    }
    if (dtype != FMM_F64 && dtype != FMM_F32) { fmm_set_error("fmm_direct_noalloc: dtype must be FMM_F64 or FMM_F32"); return FMM_ERR_ARG; }
    if (flags & ~FMM_OUT_FIELD) { fmm_set_error("fmm_direct_noalloc: only FMM_OUT_FIELD is accepted in flags"); return FMM_ERR_ARG; }
    if (n > 0 && (!pos || !q)) { fmm_set_error("fmm_direct_noalloc: pos and q must not be NULL"); return FMM_ERR_ARG; }
    if (n == 0) return FMM_OK;
    void* scratch = nullptr;
    int sms = 0;
    int rc = scratch_for_current_device(&scratch, &sms);
    if (rc) return rc;
    int field = (flags & FMM_OUT_FIELD) ? 1 : 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == FMM_F64)
        return direct_noalloc_typed<double>(n, (const double*)pos, (const double*)q, (double*)phi, (double*)force,
                                            field, st, scratch, sms);
    return direct_noalloc_typed<float>(n, (const float*)pos, (const float*)q, (float*)phi, (float*)force, field, st,
                                       scratch, sms);
}

extern "C" int64_t fmm_direct_noalloc_max_n(void) { return kNoAllocMaxN; }
