// Host-link probe: measures the link between the GPU and the host memory that
// holds the graph and the full vectors (the paper's PCIe 4.0 link, quoted at
// 32 GB/s peak in §6.1; NVLink-C2C on a Grace-hosted GB300).  Three figures:
// copy-engine bandwidth of page-locked host-to-device copies, bandwidth of a
// kernel that gathers random rows in place from mapped host memory (the
// search's own access pattern), the latency of dependent single loads, and
// the rate at which the host's own cores gather random rows into a staging
// buffer (the paper's FetchNeighbors path, Alg. 2, whose rows then cross by
// copy engine: that path moves at most the smaller of the two rates).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "bang.h"

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// Every warp reads `rounds` x 4 random rows of row_vec 16-byte words; lane i
// reads word i of a row (row_vec <= 32).  The xor of everything read goes to
// `sink` so that no load is dropped.
__global__ void gather_rows(const uint4 *__restrict__ host, uint64_t nrows, uint32_t row_vec,
                            uint32_t rounds, unsigned long long *sink)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    uint32_t acc = 0;
    for (uint32_t r = 0; r < rounds; ++r) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t row = mix64(warp * 0x9E3779B97F4A7C15ull + r * 4u + u) % nrows;
            v[u] = lane < row_vec ? host[row * row_vec + lane] : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);
}

// One thread follows a cyclic chain through host memory: next[slot * stride].
__global__ void chase(const uint32_t *__restrict__ next, uint32_t stride, uint32_t steps,
                      uint32_t *out)
{
    uint32_t i = 0;
    for (uint32_t s = 0; s < steps; ++s) i = *(volatile const uint32_t *)(next + static_cast<uint64_t>(i) * stride);
    *out = i;
}

}  // namespace

extern "C" int bang_probe_host_link(int device, uint64_t bytes, uint32_t row_bytes,
                                    bang_link_probe *out)
{
    if (!out || bytes < (1u << 20) || row_bytes == 0 || row_bytes % 16 || row_bytes > 512)
        return BANG_EINVAL;
    std::memset(out, 0, sizeof *out);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return BANG_ECUDA;
    }
    int rc = BANG_OK;
    void *h = nullptr, *dbuf = nullptr;
    uint32_t *dout = nullptr;
    unsigned long long *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    const uint32_t stride = 1024;                  // one chain slot per 4 KB
    const uint64_t nslots = bytes / (stride * 4ull);
    const uint64_t nrows = bytes / row_bytes;
    do {
        if (cudaHostAlloc(&h, bytes, cudaHostAllocMapped) != cudaSuccess) { rc = BANG_ENOMEM; break; }
        if (cudaMalloc(&dbuf, bytes) != cudaSuccess) { rc = BANG_ENOMEM; break; }
        if (cudaMalloc(&dout, sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&sink, sizeof(unsigned long long)) != cudaSuccess) { rc = BANG_ENOMEM; break; }
        std::memset(h, 1, bytes);
        {   // random cyclic permutation of the chain slots (Sattolo)
            std::vector<uint32_t> perm(nslots);
            for (uint64_t i = 0; i < nslots; ++i) perm[i] = static_cast<uint32_t>(i);
            uint64_t s = 88172645463325252ull;
            for (uint64_t i = nslots - 1; i > 0; --i) {
                s ^= s << 13; s ^= s >> 7; s ^= s << 17;
                uint64_t j = s % i;
                uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
            }
            uint32_t *nx = static_cast<uint32_t *>(h);
            for (uint64_t i = 0; i < nslots; ++i) nx[perm[i] * (uint64_t)stride] = perm[(i + 1) % nslots];
        }
        void *hd = nullptr;
        if (cudaHostGetDevicePointer(&hd, h, 0) != cudaSuccess) { rc = BANG_ECUDA; break; }
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { rc = BANG_ECUDA; break; }
        cudaMemset(sink, 0, sizeof(unsigned long long));

        double best = 0;                           // copy engine
        for (int t = 0; t < 3; ++t) {
            cudaEventRecord(e0);
            cudaMemcpyAsync(dbuf, h, bytes, cudaMemcpyHostToDevice);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms > 0 && bytes / (ms * 1e6) > best) best = bytes / (ms * 1e6);
        }
        out->h2d_copy_gbs = best;

        int sms = 0;                               // gather of random rows in place
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        const uint32_t rounds = 64, threads = 512;
        const uint32_t blocks = static_cast<uint32_t>(sms) * 4u;
        best = 0;
        for (int t = 0; t < 3; ++t) {
            cudaEventRecord(e0);
            gather_rows<<<blocks, threads>>>(static_cast<const uint4 *>(hd), nrows, row_bytes / 16,
                                             rounds, sink);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            const double moved = (double)blocks * (threads / 32) * rounds * 4 * row_bytes;
            if (ms > 0 && moved / (ms * 1e6) > best) best = moved / (ms * 1e6);
        }
        out->gather_gbs = best;
        out->gather_row_bytes = row_bytes;

        {   // host threads gathering random rows into a page-locked staging ring
            const unsigned nt = std::max(1u, std::thread::hardware_concurrency());
            const uint64_t ring_rows = 4096;       // per thread
            void *stage = nullptr;
            if (cudaHostAlloc(&stage, (size_t)nt * ring_rows * row_bytes, cudaHostAllocDefault) == cudaSuccess) {
                std::atomic<uint64_t> moved{0};
                std::vector<std::thread> th;
                const auto t0 = std::chrono::steady_clock::now();
                for (unsigned t = 0; t < nt; ++t)
                    th.emplace_back([&, t]() {
                        const uint8_t *src = static_cast<const uint8_t *>(h);
                        uint8_t *dst = static_cast<uint8_t *>(stage) + (size_t)t * ring_rows * row_bytes;
                        uint64_t s = 0x9E3779B97F4A7C15ull * (t + 1), done = 0;
                        for (int rep = 0; rep < 64; ++rep)
                            for (uint64_t r = 0; r < ring_rows; ++r) {
                                s ^= s << 13; s ^= s >> 7; s ^= s << 17;
                                std::memcpy(dst + r * row_bytes, src + (s % nrows) * row_bytes, row_bytes);
                                done += row_bytes;
                            }
                        moved += done;
                    });
                for (auto &x : th) x.join();
                const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                out->cpu_gather_gbs = sec > 0 ? (double)moved.load() / sec / 1e9 : 0.0;
                out->cpu_threads = nt;
                cudaFreeHost(stage);
            } else {
                cudaGetLastError();
            }
        }

        const uint32_t steps = 20000;              // dependent loads
        chase<<<1, 1>>>(static_cast<const uint32_t *>(hd), stride, 200, dout);
        cudaEventRecord(e0);
        chase<<<1, 1>>>(static_cast<const uint32_t *>(hd), stride, steps, dout);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        out->latency_ns = ms * 1e6 / steps;
        if (cudaGetLastError() != cudaSuccess) rc = BANG_ECUDA;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (dout) cudaFree(dout);
    if (dbuf) cudaFree(dbuf);
    if (h) cudaFreeHost(h);
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}
