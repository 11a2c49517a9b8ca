// GPU product quantisation (§4: the vector is split into M contiguous
// subspaces, the first d mod M of them one dimension wider; 256 centroids
// per subspace by k-means; a point's code is its nearest centroid in each
// subspace).  Training runs Lloyd iterations from the given initial points:
// assignment to the nearest centroid (FP64 distance summed in ascending
// dimension order, each difference, product and sum rounded; ties to the
// smaller centroid), then every centroid becomes the FP64 mean of its
// points, summed in training-sample order (a centroid with no points keeps
// its position).  Encoding uses the FP32 codebook the same way.  Every sum
// has a fixed order, so codebook and codes are the same bytes on every run.
//
// Assignment and encoding: one thread per (point, subspace), the subspace's
// centroids in shared memory.  Update: one thread per (subspace, centroid)
// scanning the assignments in sample order.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "bang.h"
#include "bang_internal.h"

namespace {

constexpr uint32_t kMaxDsub = 16;       // dimensions per subspace

struct PArgs {
    const void *X;              // n x d elements of dtype (device)
    int dtype;
    uint32_t d, M;
    const uint32_t *off;        // M + 1
    const uint64_t *sample;     // ns row ids
    uint64_t ns, n;
    double *cent;               // 256 * d, subspace s at 256 * off[s], centroid c at + c * ds
    uint8_t *asg;               // M x ns assignments
    const float *cb;            // 256 * d codebook (encode)
    uint8_t *codes;             // n x M
};

__device__ __forceinline__ double elem(const PArgs &a, uint64_t i)
{
    if (a.dtype == 0) return static_cast<double>(static_cast<const uint8_t *>(a.X)[i]);
    if (a.dtype == 1) return static_cast<double>(static_cast<const int8_t *>(a.X)[i]);
    return static_cast<double>(static_cast<const float *>(a.X)[i]);
}

// blockIdx.y = subspace; threads over the training sample.
__global__ void assign(const PArgs a)
{
    __shared__ double c[256 * kMaxDsub];            // 256 x ds doubles
    const uint32_t s = blockIdx.y, o = a.off[s], ds = a.off[s + 1] - o;
    for (uint32_t i = threadIdx.x; i < 256 * ds; i += blockDim.x) c[i] = a.cent[256ull * o + i];
    __syncthreads();
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < a.ns;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t row = a.sample[i] * a.d + o;
        double x[kMaxDsub];
        for (uint32_t j = 0; j < ds; ++j) x[j] = elem(a, row + j);
        double best = __longlong_as_double(0x7FF0000000000000ll);     // +inf
        uint32_t bc = 0;
        for (uint32_t cc = 0; cc < 256; ++cc) {
            double acc = 0.0;
            for (uint32_t j = 0; j < ds; ++j) {
                const double t = __dsub_rn(x[j], c[cc * ds + j]);
                acc = __dadd_rn(acc, __dmul_rn(t, t));
            }
            if (acc < best) { best = acc; bc = cc; }
        }
        a.asg[static_cast<uint64_t>(s) * a.ns + i] = static_cast<uint8_t>(bc);
    }
}

// One thread per (subspace, centroid): the mean of its points in sample order.
__global__ void update(const PArgs a)
{
    const uint32_t s = blockIdx.x, cc = threadIdx.x;      // 256 threads
    const uint32_t o = a.off[s], ds = a.off[s + 1] - o;
    double sum[kMaxDsub];
    for (uint32_t j = 0; j < ds; ++j) sum[j] = 0.0;
    uint64_t cnt = 0;
    const uint8_t *as = a.asg + static_cast<uint64_t>(s) * a.ns;
    for (uint64_t i = 0; i < a.ns; ++i) {
        if (as[i] != cc) continue;
        ++cnt;
        const uint64_t row = a.sample[i] * a.d + o;
        for (uint32_t j = 0; j < ds; ++j) sum[j] = __dadd_rn(sum[j], elem(a, row + j));
    }
    if (cnt == 0) return;
    double *cen = a.cent + 256ull * o + static_cast<uint64_t>(cc) * ds;
    for (uint32_t j = 0; j < ds; ++j) cen[j] = __ddiv_rn(sum[j], static_cast<double>(cnt));
}

__global__ void to_float(const double *cent, uint64_t count, float *cb)
{
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        cb[i] = __double2float_rn(cent[i]);
}

// blockIdx.y = subspace; threads over the points.
__global__ void encode(const PArgs a)
{
    __shared__ float c[256 * kMaxDsub];
    const uint32_t s = blockIdx.y, o = a.off[s], ds = a.off[s + 1] - o;
    for (uint32_t i = threadIdx.x; i < 256 * ds; i += blockDim.x) c[i] = a.cb[256ull * o + i];
    __syncthreads();
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < a.n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t row = i * a.d + o;
        double best = __longlong_as_double(0x7FF0000000000000ll);
        uint32_t bc = 0;
        for (uint32_t cc = 0; cc < 256; ++cc) {
            double acc = 0.0;
            for (uint32_t j = 0; j < ds; ++j) {
                const double t = __dsub_rn(elem(a, row + j), static_cast<double>(c[cc * ds + j]));
                acc = __dadd_rn(acc, __dmul_rn(t, t));
            }
            if (acc < best) { best = acc; bc = cc; }
        }
        a.codes[i * a.M + s] = static_cast<uint8_t>(bc);
    }
}

__global__ void init_cent(const PArgs a, const uint64_t *init)
{
    const uint32_t s = blockIdx.x, cc = threadIdx.x;
    const uint32_t o = a.off[s], ds = a.off[s + 1] - o;
    const uint64_t row = init[static_cast<uint64_t>(s) * 256 + cc] * a.d + o;
    for (uint32_t j = 0; j < ds; ++j) a.cent[256ull * o + static_cast<uint64_t>(cc) * ds + j] = elem(a, row + j);
}

template <typename T> struct DArr {
    T *p = nullptr;
    ~DArr() { if (p) cudaFree(p); }
    cudaError_t alloc(uint64_t count) { return cudaMalloc(&p, sizeof(T) * (count ? count : 1)); }
};

int pfail(int code, const std::string &m)
{
    bang::set_error(m);
    return code;
}

bool is_dev(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

#define PQ_TRY(x)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (x);                                                               \
        if (e_ != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            return pfail(e_ == cudaErrorMemoryAllocation ? BANG_ENOMEM : BANG_ECUDA,       \
                         std::string(#x) + ": " + cudaGetErrorString(e_));                  \
        }                                                                                   \
    } while (0)

extern "C" int bang_build_pq(int device, const void *base, bang_dtype dtype, uint64_t n, uint32_t d,
                             uint32_t M, const uint64_t *sample, uint64_t ns, const uint64_t *init,
                             uint32_t iters, float *codebook, uint8_t *codes, void *stream)
{
    if (!base || !sample || !init || !codebook || !codes)
        return pfail(BANG_EINVAL, "bang_build_pq: NULL argument");
    if (dtype != BANG_U8 && dtype != BANG_I8 && dtype != BANG_F32)
        return pfail(BANG_EINVAL, "bang_build_pq: unknown dtype");
    if (n == 0 || d == 0 || M == 0 || M > d || ns == 0 || iters > 1000)
        return pfail(BANG_EINVAL, "bang_build_pq: need n, d, ns > 0, 1 <= M <= d, iters <= 1000");
    if ((d + M - 1) / M > kMaxDsub) return pfail(BANG_EINVAL, "bang_build_pq: subspaces wider than 16 dimensions");
    if (bang::pointer_kind(base, device) == 2 || bang::pointer_kind(codebook, device) == 2 ||
        bang::pointer_kind(codes, device) == 2)
        return pfail(BANG_EINVAL, "bang_build_pq: base, codebook or codes is memory of another GPU");
    if (is_dev(sample) || is_dev(init)) return pfail(BANG_EINVAL, "bang_build_pq: sample and init must be host memory");
    for (uint64_t i = 0; i < ns; ++i)
        if (sample[i] >= n) return pfail(BANG_EINVAL, "bang_build_pq: sample id >= n");
    for (uint64_t i = 0; i < 256ull * M; ++i)
        if (init[i] >= n) return pfail(BANG_EINVAL, "bang_build_pq: init id >= n");
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return pfail(BANG_ECUDA, "bang_build_pq: cannot select the device");
    }
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{prev};
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    std::vector<uint32_t> off(M + 1);
    for (uint32_t s = 0, o = 0; s <= M; ++s) {        // first d mod M subspaces one wider (§6.3)
        off[s] = o;
        if (s < M) o += d / M + (s < d % M ? 1u : 0u);
    }
    const uint32_t esz = dtype == BANG_F32 ? 4u : 1u;
    DArr<uint8_t> X, asg, dcodes;
    DArr<uint32_t> doff;
    DArr<uint64_t> dsample, dinit;
    DArr<double> cent;
    DArr<float> cb;
    const void *Xd = base;
    if (!is_dev(base)) {
        PQ_TRY(X.alloc(n * d * esz));
        PQ_TRY(cudaMemcpyAsync(X.p, base, n * d * esz, cudaMemcpyHostToDevice, st));
        Xd = X.p;
    }
    PQ_TRY(doff.alloc(M + 1));
    PQ_TRY(cudaMemcpyAsync(doff.p, off.data(), (M + 1) * 4, cudaMemcpyHostToDevice, st));
    PQ_TRY(dsample.alloc(ns));
    PQ_TRY(cudaMemcpyAsync(dsample.p, sample, ns * 8, cudaMemcpyHostToDevice, st));
    PQ_TRY(dinit.alloc(256ull * M));
    PQ_TRY(cudaMemcpyAsync(dinit.p, init, 256ull * M * 8, cudaMemcpyHostToDevice, st));
    PQ_TRY(cent.alloc(256ull * d));
    PQ_TRY(cb.alloc(256ull * d));
    PQ_TRY(asg.alloc(ns * M));
    const bool codes_dev = is_dev(codes);
    if (!codes_dev) PQ_TRY(dcodes.alloc(n * M));

    PArgs a;
    std::memset(&a, 0, sizeof a);
    a.X = Xd;
    a.dtype = dtype;
    a.d = d;
    a.M = M;
    a.off = doff.p;
    a.sample = dsample.p;
    a.ns = ns;
    a.n = n;
    a.cent = cent.p;
    a.asg = asg.p;
    a.cb = cb.p;
    a.codes = codes_dev ? codes : dcodes.p;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    init_cent<<<M, 256, 0, st>>>(a, dinit.p);
    const uint32_t bx = static_cast<uint32_t>(sms) * 4u / M + 1u;
    for (uint32_t it = 0; it < iters; ++it) {
        assign<<<dim3(bx, M), 256, 0, st>>>(a);
        update<<<M, 256, 0, st>>>(a);
    }
    to_float<<<256, 256, 0, st>>>(cent.p, 256ull * d, cb.p);
    encode<<<dim3(bx * 4, M), 256, 0, st>>>(a);
    PQ_TRY(cudaGetLastError());
    PQ_TRY(cudaMemcpyAsync(codebook, cb.p, 256ull * d * 4, cudaMemcpyDefault, st));
    if (!codes_dev) PQ_TRY(cudaMemcpyAsync(codes, dcodes.p, n * M, cudaMemcpyDeviceToHost, st));
    PQ_TRY(cudaStreamSynchronize(st));
    return BANG_OK;
}
