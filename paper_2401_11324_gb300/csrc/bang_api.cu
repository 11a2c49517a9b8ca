// C ABI of the GB300 BANG search path (declarations and contracts in
// include/bang.h).  Host-side responsibilities: argument and index
// validation, device copies of the PQ data, page-locking and mapping of the
// host-resident graph and vectors (read in place by the kernel, Alg. 2's
// FetchNeighbors), staging of host queries and results, and the launch.
#include <cuda_runtime.h>
#include <sys/mman.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <map>
#include <numeric>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "bang.h"
#include "adc_table_tc.h"
#include "bang_internal.h"
#include "rerank.h"
#include "search_kernel.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            int code_ = (e_ == cudaErrorMemoryAllocation) ? BANG_ENOMEM : BANG_ECUDA;        \
            return fail(code_, "%s failed: %s", #call, cudaGetErrorString(e_));             \
        }                                                                                     \
    } while (0)

// A host range the GPU reads in place.  Registered by the library unless the
// caller's memory is already page-locked (or device-accessible already).
// Host ranges that do not start on a 128-byte boundary are replaced by an
// aligned page-locked copy owned by the index: rows of 32-byte multiples then
// start on 32-byte sector boundaries, and a 256-byte neighbour row crosses
// the host link as 8 sectors instead of 9.
constexpr uintptr_t kHostAlign = 128;

// Page-locked, mapped host memory for the library's own host copies (an
// aligned copy of a caller's array, packed rows, node records): a mapping
// advised for transparent huge pages (bang_host_alloc) registered with CUDA,
// so that the GPU's reads of it need few address translations.
cudaError_t huge_host_alloc(size_t bytes, void **out)
{
    void *p = nullptr;
    *out = nullptr;
    if (bang_host_alloc(bytes, &p) != BANG_OK) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaHostRegister(p, bytes, cudaHostRegisterMapped);
    if (e != cudaSuccess) {
        cudaGetLastError();
        bang_host_free(p);
        return e;
    }
    *out = p;
    return cudaSuccess;
}

void huge_host_free(void *p)
{
    cudaHostUnregister(p);
    bang_host_free(p);
}

struct HostView {
    const void *host = nullptr;
    const void *dev = nullptr;
    bool registered_here = false;
    bool copied = false;             // `host` is the library's aligned copy

    void release()
    {
        if (copied && host) huge_host_free(const_cast<void *>(host));
        else if (registered_here && host) cudaHostUnregister(const_cast<void *>(host));
        host = dev = nullptr;
        registered_here = copied = false;
    }
};

// memcpy split over the host's cores (the copies run once, at registration).
void parallel_copy(void *dst, const void *src, size_t bytes)
{
    const size_t chunk = size_t(64) << 20;
    unsigned nt = std::thread::hardware_concurrency();
    nt = nt ? nt : 1u;
    const size_t parts = (bytes + chunk - 1) / chunk;
    if (parts < 2 || nt < 2) {
        std::memcpy(dst, src, bytes);
        return;
    }
    nt = static_cast<unsigned>(parts < nt ? parts : nt);
    std::atomic<size_t> next{0};
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&] {
            for (size_t i; (i = next.fetch_add(1)) < parts;) {
                const size_t o = i * chunk, m = bytes - o < chunk ? bytes - o : chunk;
                std::memcpy(static_cast<char *>(dst) + o, static_cast<const char *>(src) + o, m);
            }
        });
    for (auto &t : th) t.join();
}

int map_host(const void *p, size_t bytes, int device, HostView &out)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
    }
    out.host = p;
    out.registered_here = out.copied = false;
    if (at.type == cudaMemoryTypeDevice && at.device != device)
        return fail(BANG_EINVAL, "the array is device memory of GPU %d, not of the index's GPU %d",
                    at.device, device);
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        out.dev = p;
        return BANG_OK;
    }
    if (reinterpret_cast<uintptr_t>(p) % kHostAlign != 0) {
        void *c = nullptr;
        e = huge_host_alloc(bytes, &c);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? BANG_ENOMEM : BANG_ECUDA,
                        "aligned page-locked copy of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        }
        parallel_copy(c, p, bytes);
        void *dp = nullptr;
        e = cudaHostGetDevicePointer(&dp, c, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            huge_host_free(c);
            return fail(BANG_ECUDA, "cudaHostGetDevicePointer failed: %s", cudaGetErrorString(e));
        }
        out.host = c;
        out.dev = dp;
        out.copied = true;
        return BANG_OK;
    }
    if (at.type == cudaMemoryTypeUnregistered) {
        e = cudaHostRegister(const_cast<void *>(p), bytes,
                             cudaHostRegisterMapped | cudaHostRegisterReadOnly);
        if (e != cudaSuccess) {
            cudaGetLastError();
            // some systems refuse the read-only flag; retry without it
            e = cudaHostRegister(const_cast<void *>(p), bytes, cudaHostRegisterMapped);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? BANG_ENOMEM : BANG_ECUDA,
                        "cudaHostRegister of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        }
        out.registered_here = true;
    }
    void *dp = nullptr;
    e = cudaHostGetDevicePointer(&dp, const_cast<void *>(p), 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (out.registered_here) cudaHostUnregister(const_cast<void *>(p));
        out.registered_here = false;
        return fail(BANG_ECUDA, "cudaHostGetDevicePointer failed: %s", cudaGetErrorString(e));
    }
    out.dev = dp;
    return BANG_OK;
}

// Where a caller's pointer lives: host memory (pageable or page-locked),
// device memory of `device` (or managed memory, reachable from every GPU),
// or device memory of another GPU, which the index's kernels must not be
// given: without peer access that is a fault on that GPU.
enum PtrKind { kPtrHost = 0, kPtrDevice = 1, kPtrOtherDevice = 2 };

PtrKind pointer_kind(const void *p, int device)
{
    if (!p) return kPtrHost;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return kPtrHost;
    }
    if (at.type == cudaMemoryTypeManaged) return kPtrDevice;
    if (at.type == cudaMemoryTypeDevice) return at.device == device ? kPtrDevice : kPtrOtherDevice;
    return kPtrHost;
}

bool is_device_accessible(const void *p, int device) { return pointer_kind(p, device) == kPtrDevice; }

size_t elem_size(int dt) { return dt == BANG_F32 ? 4 : 1; }

// Device buffer that only grows.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t want)
    {
        if (want <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) bytes = want;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

}  // namespace

namespace bang {
void set_error(const std::string &msg) { g_err = msg; }
int pointer_kind(const void *p, int device) { return ::pointer_kind(p, device); }
}  // namespace bang

struct bang_index {
    int device = 0;
    uint32_t d = 0, M = 0, Mpad = 0, R = 0, medoid = 0;
    uint64_t n = 0;
    int dtype = -1;
    float *codebook = nullptr;
    uint32_t *off = nullptr;
    uint8_t *codes = nullptr;
    HostView adj, base;
    // Packed graph rows (BANG_GRAPH_PACKED): ids of adj_bits bits, rows of
    // adj_row_words words, page-locked and owned by the index.
    HostView adj_packed;
    uint32_t adj_bits = 0, adj_row_words = 0;
    // Node records (BANG_NODE_RECORDS): each node's row (packed or not) and
    // full vector side by side, rec_words words per node (a multiple of 8),
    // page-locked and owned by the index.
    HostView records;
    uint32_t rec_words = 0, rec_row_words = 0;
    bool rec_packed = false;
    bool have_pq = false, have_graph = false, have_vectors = false;
    DevBuf staging;
    // In-memory placement (§5.1): device copies of the graph and/or vectors.
    DevBuf adj_hbm, base_hbm;
    // Neighbour-code layout (BANG_NEIGHBOR_CODES): for every node the code
    // rows of its R neighbours, 32 bytes each, in HBM.
    DevBuf ncodes;
    bool ncodes_ok = false;
    uint32_t placement = 0;
    // Batched form: per-stream work counter, query order and staged k / L.
    std::map<cudaStream_t, DevBuf> work;
    // Tensor-core tables: centroid tiles (BF16 hi/lo, core-matrix layout),
    // first tile per subspace, squared centroid norms; per-stream table
    // scratch for searches that read precomputed tables; error flag.
    DevBuf tc_btiles, tc_bfirst, tc_cnorm, tc_err;
    DevBuf tc_btiles_tf32;    // the same tiles with the centroids rounded to TF32
    bool tc_ok = false;
    std::map<cudaStream_t, DevBuf> tables;
    // Staged re-rank: per-stream candidate lists (nq rows of the iteration
    // cap) and their lengths.
    std::map<cudaStream_t, DevBuf> cands;
};

namespace bang {
int index_device(const bang_index *ix) { return ix->device; }
uint32_t index_placement(const bang_index *ix) { return ix->placement; }
}  // namespace bang

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
        else cudaGetLastError();
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Round-to-nearest-even FP32 -> BF16 (finite inputs).
uint16_t bf16_rne(float x)
{
    uint32_t b;
    std::memcpy(&b, &x, 4);
    b += 0x7FFFu + ((b >> 16) & 1u);
    return static_cast<uint16_t>(b >> 16);
}
float bf16_to_f32(uint16_t h)
{
    const uint32_t b = static_cast<uint32_t>(h) << 16;
    float x;
    std::memcpy(&x, &b, 4);
    return x;
}

// Centroid operands of the tensor-core table kernel: for every subspace and
// every 16-wide K block it touches, a 256 x 16 BF16 tile of the centroids
// (zero outside the subspace's dimensions) in the no-swizzle K-major
// core-matrix layout, split into high, middle and low BF16 parts.
// Round to TF32 (10 mantissa bits), to nearest with ties to even.
float tf32_rne_host(float x)
{
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0xFFFu + ((u >> 13) & 1u);
    u &= ~0x1FFFu;
    float y;
    std::memcpy(&y, &u, 4);
    return y;
}

// Centroid tiles of the tensor-core tables: per 16-dimension block three BF16
// parts of every centroid value (hi, mid, lo: about FP32), or, for the TF32
// form, the value rounded to TF32 as two exact BF16 parts and a zero part.
bool build_tc_tiles(const float *codebook, uint32_t d, uint32_t M, const std::vector<uint32_t> &off,
                    std::vector<uint16_t> &tiles, std::vector<uint32_t> &first, std::vector<float> &cnorm,
                    bool tf32 = false)
{
    const uint32_t elems = 256u * 16u;                  // one tile
    first.assign(M, 0);
    cnorm.assign((size_t)M * 256, 0.0f);
    tiles.clear();
    for (uint32_t s = 0; s < M; ++s) {
        const uint32_t o = off[s], ds = off[s + 1] - o;
        const uint32_t kb0 = o / 16, kb1 = (o + ds - 1) / 16;
        if (kb1 - kb0 + 1 > bang::kMaxKbPerSub) return false;
        first[s] = static_cast<uint32_t>(tiles.size() / elems);
        const float *cb = codebook + (size_t)256 * o;
        for (uint32_t c = 0; c < 256; ++c) {
            double acc = 0.0;
            for (uint32_t j = 0; j < ds; ++j) acc += (double)cb[c * ds + j] * (double)cb[c * ds + j];
            cnorm[(size_t)s * 256 + c] = static_cast<float>(acc);
        }
        for (uint32_t kb = kb0; kb <= kb1; ++kb) {
            const size_t base = tiles.size();
            tiles.resize(base + 3 * (size_t)elems, 0);
            for (uint32_t c = 0; c < 256; ++c)
                for (uint32_t kk = 0; kk < 16; ++kk) {
                    const uint32_t j = kb * 16 + kk;
                    float x = (j >= o && j < o + ds) ? cb[c * ds + (j - o)] : 0.0f;
                    if (tf32) x = tf32_rne_host(x);
                    const uint16_t hi = bf16_rne(x);
                    const float r1 = x - bf16_to_f32(hi);
                    const uint16_t mid = bf16_rne(r1);
                    const uint16_t lo = tf32 ? 0 : bf16_rne(r1 - bf16_to_f32(mid));
                    const size_t e = (((c >> 3) * 2 + (kk >> 3)) * 128 + (c & 7) * 16 + (kk & 7) * 2) / 2;
                    tiles[base + e] = hi;
                    tiles[base + elems + e] = mid;
                    tiles[base + 2 * (size_t)elems + e] = lo;
                }
        }
    }
    return true;
}

std::vector<uint32_t> chunk_offsets(uint32_t d, uint32_t M)
{
    std::vector<uint32_t> off(M + 1);
    uint32_t base = d / M, extra = d % M;
    off[0] = 0;
    for (uint32_t s = 0; s < M; ++s) off[s + 1] = off[s] + base + (s < extra ? 1u : 0u);
    return off;
}

// Check every row of the adjacency: ids < n, no self loop, no duplicate.
// Rows are split across host threads.
bool validate_graph(const uint32_t *adj, uint64_t n, uint32_t R, uint64_t *bad_row)
{
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<uint64_t> bad(nt, UINT64_MAX);
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) {
        th.emplace_back([&, t]() {
            uint32_t tmp[bang::kMaxR];
            uint64_t lo = n * t / nt, hi = n * (t + 1) / nt;
            for (uint64_t i = lo; i < hi; ++i) {
                const uint32_t *row = adj + i * R;
                uint32_t m = 0;
                for (uint32_t r = 0; r < R; ++r) {
                    uint32_t v = row[r];
                    if (v == bang::kNone) continue;
                    if (v >= n || v == i) { bad[t] = i; return; }
                    tmp[m++] = v;
                }
                std::sort(tmp, tmp + m);
                for (uint32_t r = 1; r < m; ++r)
                    if (tmp[r] == tmp[r - 1]) { bad[t] = i; return; }
            }
        });
    }
    for (auto &x : th) x.join();
    for (unsigned t = 0; t < nt; ++t)
        if (bad[t] != UINT64_MAX) { *bad_row = bad[t]; return false; }
    return true;
}

// Packs the registered rows: b = the fewest bits with 2^b - 1 >= n (the
// all-ones value marks an empty slot), rows rounded up to 8 words (32 bytes)
// so that every row starts on a sector boundary.
int build_packed_rows(bang_index *ix)
{
    if (ix->adj_packed.host) return BANG_OK;
    uint32_t b = 1;
    while (((1ull << b) - 1ull) < ix->n) ++b;
    if (b > 31) return fail(BANG_EINVAL, "bang_set_placement: ids need more than 31 bits");
    const uint32_t words = ((ix->R * b + 31u) / 32u + 7u) & ~7u;
    const size_t bytes = (size_t)ix->n * words * 4u;
    void *h = nullptr;
    cudaError_t e = huge_host_alloc(bytes, &h);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BANG_ENOMEM, "packed graph rows: %zu bytes of page-locked memory: %s", bytes,
                    cudaGetErrorString(e));
    }
    const uint32_t *src = static_cast<const uint32_t *>(ix->adj.host);
    const uint64_t n = ix->n;
    const uint32_t R = ix->R, mask = (1u << b) - 1u;
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([=]() {
            for (uint64_t i = n * t / nt; i < n * (t + 1) / nt; ++i) {
                uint32_t *out = static_cast<uint32_t *>(h) + i * words;
                std::memset(out, 0, words * 4u);
                for (uint32_t r = 0; r < R; ++r) {
                    const uint32_t v = src[i * R + r] == bang::kNone ? mask : src[i * R + r];
                    const uint64_t bit = (uint64_t)r * b;
                    const uint32_t wi = (uint32_t)(bit >> 5), o = (uint32_t)(bit & 31u);
                    out[wi] |= v << o;
                    if (o + b > 32u) out[wi + 1] |= v >> (32u - o);
                }
            }
        });
    for (auto &x : th) x.join();
    void *dp = nullptr;
    e = cudaHostGetDevicePointer(&dp, h, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        huge_host_free(h);
        return fail(BANG_ECUDA, "cudaHostGetDevicePointer failed: %s", cudaGetErrorString(e));
    }
    ix->adj_packed.host = h;
    ix->adj_packed.dev = dp;
    ix->adj_packed.copied = true;
    ix->adj_bits = b;
    ix->adj_row_words = words;
    return BANG_OK;
}

// One thread per (node, slot): the slot's neighbour's code row (zeros for an
// empty slot), padded to 32 bytes.
__global__ void gather_neighbor_codes(const uint32_t *adj, uint64_t n, uint32_t R, const uint8_t *codes,
                                      uint32_t Mpad, uint4 *out)
{
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < n * R;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t id = adj[e];
        uint4 c0 = make_uint4(0u, 0u, 0u, 0u), c1 = c0;
        if (id != bang::kNone) {
            const uint4 *src = reinterpret_cast<const uint4 *>(codes + static_cast<uint64_t>(id) * Mpad);
            c0 = src[0];
            if (Mpad > 16u) c1 = src[1];
        }
        out[2 * e] = c0;
        out[2 * e + 1] = c1;
    }
}

// Where and how the kernel reads the graph rows.
// Builds the node records: row i (packed when `packed`) then vector i, the
// record rounded up to 32 bytes so that every record starts on a sector.
int build_records(bang_index *ix, bool packed)
{
    if (ix->records.host && ix->rec_packed == packed) return BANG_OK;
    ix->records.release();
    if (packed) {
        const int rc = build_packed_rows(ix);
        if (rc) return rc;
    }
    const uint32_t rw = packed ? ix->adj_row_words : ix->R;
    const size_t vb = (size_t)ix->d * elem_size(ix->dtype);
    const uint32_t words = (uint32_t)((((size_t)rw * 4u + vb + 31u) / 32u) * 8u);
    const size_t bytes = (size_t)ix->n * words * 4u;
    void *h = nullptr;
    cudaError_t e = huge_host_alloc(bytes, &h);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BANG_ENOMEM, "node records: %zu bytes of page-locked memory: %s", bytes,
                    cudaGetErrorString(e));
    }
    const unsigned char *rows = static_cast<const unsigned char *>(packed ? ix->adj_packed.host : ix->adj.host);
    const unsigned char *vec = static_cast<const unsigned char *>(ix->base.host);
    const uint64_t n = ix->n;
    const size_t rb = (size_t)rw * 4u, recb = (size_t)words * 4u;
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([=]() {
            for (uint64_t i = n * t / nt; i < n * (t + 1) / nt; ++i) {
                unsigned char *out = static_cast<unsigned char *>(h) + i * recb;
                std::memcpy(out, rows + i * rb, rb);
                std::memcpy(out + rb, vec + i * vb, vb);
                std::memset(out + rb + vb, 0, recb - rb - vb);
            }
        });
    for (auto &x : th) x.join();
    void *dp = nullptr;
    e = cudaHostGetDevicePointer(&dp, h, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        huge_host_free(h);
        return fail(BANG_ECUDA, "cudaHostGetDevicePointer failed: %s", cudaGetErrorString(e));
    }
    ix->records.host = h;
    ix->records.dev = dp;
    ix->records.copied = true;
    ix->rec_words = words;
    ix->rec_row_words = rw;
    ix->rec_packed = packed;
    return BANG_OK;
}

// Where the search reads rows and vectors, and their strides.
void set_graph_args(const bang_index *ix, bang::SearchArgs &a)
{
    a.ncodes = (ix->placement & BANG_NEIGHBOR_CODES) ? static_cast<const uint8_t *>(ix->ncodes.p) : nullptr;
    const bool pk = (ix->placement & BANG_GRAPH_PACKED) != 0;
    a.adj_bits = pk ? ix->adj_bits : 0u;
    a.adj_row_words = pk ? ix->adj_row_words : ix->R;
    if (ix->placement & BANG_NODE_RECORDS) {
        const uint32_t *rec = static_cast<const uint32_t *>(ix->records.dev);
        a.adj = rec;
        a.adj_stride = ix->rec_words;
        a.base = rec + ix->rec_row_words;
        a.vstride = ix->rec_words * 4u / (uint32_t)elem_size(ix->dtype);
        return;
    }
    if (ix->placement & BANG_GRAPH_IN_HBM) a.adj = static_cast<const uint32_t *>(ix->adj_hbm.p);
    else a.adj = static_cast<const uint32_t *>(pk ? ix->adj_packed.dev : ix->adj.dev);
    a.adj_stride = a.adj_row_words;
    a.base = (ix->placement & BANG_VECTORS_IN_HBM) ? ix->base_hbm.p : ix->base.dev;
    a.vstride = ix->d;
}

}  // namespace

extern "C" {

const char *bang_last_error(void) { return g_err.c_str(); }

int bang_create(int device, bang_index **out)
{
    if (!out) return fail(BANG_EINVAL, "bang_create: out is NULL");
    *out = nullptr;
    int count = 0;
    CUDA_TRY(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count)
        return fail(BANG_EINVAL, "bang_create: device %d not in [0, %d)", device, count);
    bang_index *ix = new (std::nothrow) bang_index();
    if (!ix) return fail(BANG_ENOMEM, "bang_create: out of host memory");
    ix->device = device;
    *out = ix;
    return BANG_OK;
}

int bang_load_pq(bang_index *ix, uint32_t d, uint32_t M, const float *codebook,
                 const uint8_t *codes, uint64_t n)
{
    if (!ix || !codebook || !codes) return fail(BANG_EINVAL, "bang_load_pq: NULL argument");
    if (d == 0 || d > (uint32_t)bang::kMaxD)
        return fail(BANG_EINVAL, "bang_load_pq: d=%u outside 1..%d", d, bang::kMaxD);
    if (M == 0 || M > d || M > (uint32_t)bang::kMaxM)
        return fail(BANG_EINVAL, "bang_load_pq: M=%u outside 1..min(d, %d)", M, bang::kMaxM);
    if (n == 0 || n >= (1ull << 31)) return fail(BANG_EINVAL, "bang_load_pq: n=%llu outside 1..2^31-1",
                                                 (unsigned long long)n);
    DeviceGuard g(ix->device);
    if (!g.ok) return fail(BANG_ECUDA, "cannot select device %d", ix->device);
    if (ix->codebook) cudaFree(ix->codebook);
    if (ix->off) cudaFree(ix->off);
    if (ix->codes) cudaFree(ix->codes);
    ix->codebook = nullptr; ix->off = nullptr; ix->codes = nullptr;
    ix->ncodes.release();
    ix->ncodes_ok = false;
    ix->records.release();
    ix->placement &= ~(uint32_t)(BANG_NEIGHBOR_CODES | BANG_NODE_RECORDS);
    ix->adj.release();
    ix->base.release();
    ix->have_pq = ix->have_graph = ix->have_vectors = false;

    const uint32_t Mpad = (M + 15u) & ~15u;
    std::vector<uint32_t> off = chunk_offsets(d, M);
    CUDA_TRY(cudaMalloc(&ix->codebook, sizeof(float) * 256u * d));
    CUDA_TRY(cudaMalloc(&ix->off, sizeof(uint32_t) * (M + 1)));
    CUDA_TRY(cudaMalloc(&ix->codes, (size_t)n * Mpad));
    CUDA_TRY(cudaMemcpy(ix->codebook, codebook, sizeof(float) * 256u * d, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(ix->off, off.data(), sizeof(uint32_t) * (M + 1), cudaMemcpyHostToDevice));
    if (Mpad != M) CUDA_TRY(cudaMemset(ix->codes, 0, (size_t)n * Mpad));
    CUDA_TRY(cudaMemcpy2D(ix->codes, Mpad, codes, M, M, n, cudaMemcpyHostToDevice));
    ix->d = d; ix->M = M; ix->Mpad = Mpad; ix->n = n;
    {   // operands of the tensor-core table kernel
        std::vector<uint16_t> tiles;
        std::vector<uint32_t> first;
        std::vector<float> cn;
        ix->tc_ok = build_tc_tiles(codebook, d, M, off, tiles, first, cn) &&
                    bang::tc_table_smem_bytes(d, 2) <= 227u * 1024u;
        if (ix->tc_ok) {
            std::vector<uint16_t> tiles32;
            std::vector<uint32_t> first32;
            std::vector<float> cn32;
            build_tc_tiles(codebook, d, M, off, tiles32, first32, cn32, true);
            CUDA_TRY(ix->tc_btiles_tf32.ensure(tiles32.size() * 2));
            CUDA_TRY(cudaMemcpy(ix->tc_btiles_tf32.p, tiles32.data(), tiles32.size() * 2, cudaMemcpyHostToDevice));
            CUDA_TRY(ix->tc_btiles.ensure(tiles.size() * 2));
            CUDA_TRY(ix->tc_bfirst.ensure(first.size() * 4));
            CUDA_TRY(ix->tc_cnorm.ensure(cn.size() * 4));
            CUDA_TRY(ix->tc_err.ensure(256));
            CUDA_TRY(cudaMemcpy(ix->tc_btiles.p, tiles.data(), tiles.size() * 2, cudaMemcpyHostToDevice));
            CUDA_TRY(cudaMemcpy(ix->tc_bfirst.p, first.data(), first.size() * 4, cudaMemcpyHostToDevice));
            CUDA_TRY(cudaMemcpy(ix->tc_cnorm.p, cn.data(), cn.size() * 4, cudaMemcpyHostToDevice));
            CUDA_TRY(cudaMemset(ix->tc_err.p, 0, 256));
        }
    }
    ix->have_pq = true;
    return BANG_OK;
}

int bang_register_graph(bang_index *ix, const uint32_t *adj, uint32_t R, uint32_t medoid)
{
    if (!ix || !adj) return fail(BANG_EINVAL, "bang_register_graph: NULL argument");
    if (!ix->have_pq) return fail(BANG_ESTATE, "bang_register_graph: load the PQ data first");
    if (R == 0 || R > (uint32_t)bang::kMaxR)
        return fail(BANG_EINVAL, "bang_register_graph: R=%u outside 1..%d", R, bang::kMaxR);
    if (medoid >= ix->n) return fail(BANG_EINVAL, "bang_register_graph: medoid %u >= n", medoid);
    uint64_t bad = 0;
    if (!validate_graph(adj, ix->n, R, &bad))
        return fail(BANG_EINVAL, "bang_register_graph: row %llu has an id >= n, a self loop or a "
                    "duplicate", (unsigned long long)bad);
    DeviceGuard g(ix->device);
    if (!g.ok) return fail(BANG_ECUDA, "cannot select device %d", ix->device);
    ix->adj.release();
    ix->adj_hbm.release();
    ix->adj_packed.release();
    ix->adj_bits = ix->adj_row_words = 0;
    ix->records.release();
    ix->ncodes.release();
    ix->ncodes_ok = false;
    ix->placement &= ~(uint32_t)(BANG_GRAPH_IN_HBM | BANG_GRAPH_PACKED | BANG_NEIGHBOR_CODES | BANG_NODE_RECORDS);
    ix->have_graph = false;
    int rc = map_host(adj, (size_t)ix->n * R * sizeof(uint32_t), ix->device, ix->adj);
    if (rc) return rc;
    ix->R = R;
    ix->medoid = medoid;
    ix->have_graph = true;
    return BANG_OK;
}

int bang_register_vectors(bang_index *ix, const void *base, bang_dtype dtype)
{
    if (!ix || !base) return fail(BANG_EINVAL, "bang_register_vectors: NULL argument");
    if (!ix->have_pq) return fail(BANG_ESTATE, "bang_register_vectors: load the PQ data first");
    if (dtype != BANG_U8 && dtype != BANG_I8 && dtype != BANG_F32)
        return fail(BANG_EINVAL, "bang_register_vectors: unknown dtype %d", (int)dtype);
    DeviceGuard g(ix->device);
    if (!g.ok) return fail(BANG_ECUDA, "cannot select device %d", ix->device);
    ix->base.release();
    ix->base_hbm.release();
    ix->records.release();
    ix->placement &= ~(uint32_t)(BANG_VECTORS_IN_HBM | BANG_NODE_RECORDS);
    ix->have_vectors = false;
    int rc = map_host(base, (size_t)ix->n * ix->d * elem_size(dtype), ix->device, ix->base);
    if (rc) return rc;
    ix->dtype = dtype;
    ix->have_vectors = true;
    return BANG_OK;
}

}  // extern "C"

namespace {

// Shared by bang_search (k_arr, L_arr null: every query uses k, L) and
// bang_search_batched (k, L are the bounds; persistent launch).
int search_impl(bang_index *ix, const void *queries, uint32_t nq, uint32_t k, uint32_t L,
                const uint32_t *k_arr, const uint32_t *L_arr, bool persistent,
                const bang_search_params *params, uint32_t *out_ids, float *out_dist, void *stream)
{
    if (!ix) return fail(BANG_EINVAL, "bang_search: index is NULL");
    if (!ix->have_pq || !ix->have_graph || !ix->have_vectors)
        return fail(BANG_ESTATE, "bang_search: PQ data, graph and vectors must all be set");
    if (k == 0 || k > (uint32_t)bang::kMaxK)
        return fail(BANG_EINVAL, "bang_search: k=%u outside 1..%d", k, bang::kMaxK);
    if (L < k || L > (uint32_t)bang::kMaxL)
        return fail(BANG_EINVAL, "bang_search: L=%u must satisfy k <= L <= %d", L, bang::kMaxL);
    if (nq == 0) return BANG_OK;
    if (!queries || !out_ids || !out_dist) return fail(BANG_EINVAL, "bang_search: NULL buffer");
    bang_search_params p;
    std::memset(&p, 0, sizeof p);
    if (params) p = *params;
    uint32_t log2z = p.bloom_log2 ? p.bloom_log2 : 16u;
    if (log2z < 10 || log2z > 20)
        return fail(BANG_EINVAL, "bang_search: bloom_log2=%u outside 10..20", log2z);
    if (persistent && (!k_arr || !L_arr)) return fail(BANG_EINVAL, "bang_search_batched: NULL k or L array");
    if (p.trace && p.trace_cap == 0) return fail(BANG_EINVAL, "bang_search: trace_cap is 0");

    if (p.mode > 3) return fail(BANG_EINVAL, "bang_search: unknown mode %u", p.mode);
    if (p.rerank > 2) return fail(BANG_EINVAL, "bang_search: unknown rerank %u", p.rerank);
    if (p.rerank != 0 && p.mode == 2)
        return fail(BANG_EINVAL, "bang_search: mode 2 (exact distances) has no re-rank to stage");
    if (p.smem_carveout > 100) return fail(BANG_EINVAL, "bang_search: smem_carveout %u above 100", p.smem_carveout);
    if (p.table_source == 3 && p.mode != 0)
        return fail(BANG_EINVAL, "bang_search: table_source 3 (no table) needs mode 0");
    const bool lazy = p.table_source == 3;
    const uint32_t ntab = lazy ? std::min(p.table_subspaces, ix->M) : 0u;
    bang::SmemLayout lay(ix->M, log2z, L, k, ix->d, ix->R, lazy ? (int)bang::kModeF32Lazy : (int)p.mode, ntab);
    if (lay.total > 227u * 1024u)
        return fail(BANG_EINVAL, "bang_search: %u bytes of shared memory per query exceed 227 KB "
                    "(reduce L, k, M or bloom_log2)", lay.total);

    DeviceGuard g(ix->device);
    if (!g.ok) return fail(BANG_ECUDA, "cannot select device %d", ix->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // Host buffers are staged through one device allocation.
    const size_t qbytes = (size_t)nq * ix->d * elem_size(ix->dtype);
    struct Slot { const void *user; size_t bytes; bool in; size_t off; bool dev; };
    Slot slots[10] = {
        {queries, qbytes, true, 0, false},
        {out_ids, (size_t)nq * k * 4, false, 0, false},
        {out_dist, (size_t)nq * k * 4, false, 0, false},
        {p.out_iters, (size_t)nq * 4, false, 0, false},
        {p.out_status, (size_t)nq * 4, false, 0, false},
        {p.out_ndist, (size_t)nq * 4, false, 0, false},
        {p.trace, (size_t)nq * p.trace_cap * 4, false, 0, false},
        {p.out_phase_cycles, (size_t)nq * bang::kPhases * 8, false, 0, false},
        {k_arr, (size_t)nq * 4, true, 0, false},
        {L_arr, (size_t)nq * 4, true, 0, false}};
    size_t need = 0;
    bool any_host = false;
    for (int i = 0; i < 10; ++i) {
        Slot &s = slots[i];
        if (!s.user) continue;
        const PtrKind kind = pointer_kind(s.user, ix->device);
        if (kind == kPtrOtherDevice)
            return fail(BANG_EINVAL, "bang_search: a buffer is device memory of another GPU than "
                        "the index's device %d", ix->device);
        s.dev = kind == kPtrDevice;
        if (!s.dev) {
            s.off = need;
            need += (s.bytes + 255) & ~size_t(255);
            any_host = true;
        }
    }
    if (need) CUDA_TRY(ix->staging.ensure(need));
    auto dptr = [&](int i) -> void * {
        Slot &s = slots[i];
        if (!s.user) return nullptr;
        return s.dev ? const_cast<void *>(s.user) : static_cast<char *>(ix->staging.p) + s.off;
    };
    for (int i = 0; i < 10; ++i)
        if (slots[i].user && slots[i].in && !slots[i].dev)
            CUDA_TRY(cudaMemcpyAsync(dptr(i), slots[i].user, slots[i].bytes, cudaMemcpyHostToDevice, st));

    // Persistent launch: a zeroed work counter, and, when the worklist sizes
    // are on the host, the queries ordered by decreasing L so the longest
    // searches start first.
    // Tensor-core tables (reduced-precision form): all tables of the batch
    // into per-stream scratch, then the search reads them.
    const void *tables = nullptr;
    if (p.table_source == 1 || p.table_source == 2) {
        if (p.mode != 0 && p.mode != 1)
            return fail(BANG_EINVAL, "bang_search: table_source %u needs mode 0 (FP32 tables) or 1 (BF16)",
                        p.table_source);
        if (!ix->tc_ok) return fail(BANG_EINVAL, "bang_search: tensor-core tables unavailable for this "
                                    "PQ layout (a subspace spans more than %u 16-dim blocks)", bang::kMaxKbPerSub);
        DevBuf &tb = ix->tables[st];
        CUDA_TRY(tb.ensure((size_t)nq * ix->M * 256 * (p.mode == 1 ? 2 : 4)));
        CUDA_TRY(cudaMemsetAsync(ix->tc_err.p, 0, 4, st));
        bang::TcTableArgs ta;
        ta.queries = dptr(0);
        ta.nq = nq; ta.d = ix->d; ta.M = ix->M;
        ta.off = ix->off;
        ta.btiles = static_cast<const unsigned char *>(p.table_source == 2 ? ix->tc_btiles_tf32.p : ix->tc_btiles.p);
        ta.bfirst = static_cast<const uint32_t *>(ix->tc_bfirst.p);
        ta.cnorm = static_cast<const float *>(ix->tc_cnorm.p);
        ta.out = tb.p;
        ta.out_bf16 = p.mode == 1 ? 1u : 0u;
        ta.tf32 = p.table_source == 2 ? 1u : 0u;
        ta.err = static_cast<unsigned int *>(ix->tc_err.p);
        cudaError_t te = bang::launch_tc_tables(ta, ix->dtype, st);
        if (te != cudaSuccess) return fail(BANG_ECUDA, "table kernel launch failed: %s", cudaGetErrorString(te));
        tables = tb.p;
    } else if (p.table_source != 0 && p.table_source != 3) {
        return fail(BANG_EINVAL, "bang_search: unknown table_source %u", p.table_source);
    }

    unsigned int *queue = nullptr;
    const uint32_t *order = nullptr;
    if (persistent) {
        const bool host_order = !slots[9].dev;
        DevBuf &wb = ix->work[st];
        CUDA_TRY(wb.ensure(256 + (host_order ? (size_t)nq * 4 : 0)));
        queue = static_cast<unsigned int *>(wb.p);
        CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(unsigned int), st));
        if (host_order) {
            std::vector<uint32_t> ord(nq);
            std::iota(ord.begin(), ord.end(), 0u);
            std::stable_sort(ord.begin(), ord.end(),
                             [&](uint32_t x, uint32_t y) { return L_arr[x] > L_arr[y]; });
            uint32_t *dord = reinterpret_cast<uint32_t *>(static_cast<char *>(wb.p) + 256);
            CUDA_TRY(cudaMemcpyAsync(dord, ord.data(), (size_t)nq * 4, cudaMemcpyHostToDevice, st));
            CUDA_TRY(cudaStreamSynchronize(st));      // `ord` is freed on return
            order = dord;
        }
    }

    bang::SearchArgs a;
    std::memset(&a, 0, sizeof a);
    a.queries = dptr(0);
    a.codebook = ix->codebook;
    a.off = ix->off;
    a.codes = ix->codes;
    set_graph_args(ix, a);
    a.n = (uint32_t)ix->n; a.d = ix->d; a.M = ix->M; a.Mpad = ix->Mpad; a.R = ix->R;
    a.medoid = ix->medoid;
    a.nq = nq; a.k = k; a.L = L; a.log2z = log2z; a.iter_cap = p.iter_cap;
    a.k_per_q = static_cast<const uint32_t *>(dptr(8));
    a.L_per_q = static_cast<const uint32_t *>(dptr(9));
    a.order = order;
    a.queue = queue;
    a.grid_mult = p.grid_mult;
    a.spec = p.prefetch_depth >= 2 ? 1u : 0u;
    a.early_codes = p.early_codes ? 1u : 0u;
    a.tables = tables;
    a.tables_err = static_cast<const unsigned int *>(ix->tc_err.p);
    a.out_ids = static_cast<uint32_t *>(dptr(1));
    a.out_dist = static_cast<float *>(dptr(2));
    a.out_iters = static_cast<uint32_t *>(dptr(3));
    a.out_status = static_cast<int32_t *>(dptr(4));
    a.out_ndist = static_cast<uint32_t *>(dptr(5));
    a.trace = static_cast<uint32_t *>(dptr(6));
    a.trace_cap = p.trace_cap;
    a.phase_cycles = static_cast<unsigned long long *>(dptr(7));
    a.carveout = p.smem_carveout;
    a.ntab = ntab;
    if (p.rerank != 0) {       // staged re-rank: lists sized by the iteration cap (or L)
        uint64_t cap = p.iter_cap ? p.iter_cap : 8ull * L + 64ull;
        if (cap < L) cap = L;
        const size_t lists = ((size_t)nq * cap * 4 + 255) & ~size_t(255);
        DevBuf &cb = ix->cands[st];
        CUDA_TRY(cb.ensure(lists + (size_t)nq * 4));
        a.cand = static_cast<uint32_t *>(cb.p);
        a.cand_cap = (uint32_t)cap;
        a.cand_n = reinterpret_cast<uint32_t *>(static_cast<char *>(cb.p) + lists);
        a.cand_list = p.rerank == 2 ? 1u : 0u;
    }

    {
        // 4-element vector loads need rows that start on 16-byte boundaries
        const uintptr_t qa = reinterpret_cast<uintptr_t>(a.queries);
        const uintptr_t ba = reinterpret_cast<uintptr_t>(a.base);
        a.vec_ok = (ix->d % 4 == 0) && (qa % 16 == 0) ? 1u : 0u;
        a.vecb_ok = (ix->d % 4 == 0) && (ba % 16 == 0) ? 1u : 0u;
    }
    cudaError_t le;
    if (lazy) le = bang::launch_search_f32lazy(a, ix->dtype, lay.total, st);
    else if (p.mode == 0) le = bang::launch_search_f32(a, ix->dtype, lay.total, st);
    else if (p.mode == 1) le = bang::launch_search_bf16(a, ix->dtype, lay.total, st);
    else if (p.mode == 3) le = bang::launch_search_q8(a, ix->dtype, lay.total, st);
    else le = bang::launch_search_exact(a, ix->dtype, lay.total, st);
    if (le != cudaSuccess) return fail(BANG_ECUDA, "search kernel launch failed: %s", cudaGetErrorString(le));
    if (a.cand) {
        bang::RerankArgs ra;
        std::memset(&ra, 0, sizeof ra);
        ra.queries = a.queries;
        ra.base = a.base;
        ra.vstride = a.vstride;
        ra.d = a.d;
        ra.vec_ok = a.vec_ok;
        ra.vecb_ok = a.vecb_ok;
        ra.cand = a.cand;
        ra.cand_cap = a.cand_cap;
        ra.cand_n = a.cand_n;
        ra.nq = nq; ra.k = k; ra.L = L;
        ra.k_per_q = a.k_per_q;
        ra.L_per_q = a.L_per_q;
        ra.out_ids = a.out_ids;
        ra.out_dist = a.out_dist;
        le = bang::launch_rerank(ra, ix->dtype, st);
        if (le != cudaSuccess) return fail(BANG_ECUDA, "re-rank kernel launch failed: %s", cudaGetErrorString(le));
    }
    for (int i = 1; i < 8; ++i) {
        Slot &s = slots[i];
        if (s.user && !s.dev && !s.in)
            CUDA_TRY(cudaMemcpyAsync(const_cast<void *>(s.user), dptr(i), s.bytes,
                                     cudaMemcpyDeviceToHost, st));
    }
    if (any_host) CUDA_TRY(cudaStreamSynchronize(st));
    return BANG_OK;
}

}  // namespace

extern "C" {

int bang_search(bang_index *ix, const void *queries, uint32_t nq, uint32_t k, uint32_t L,
                const bang_search_params *params, uint32_t *out_ids, float *out_dist,
                void *stream)
{
    return search_impl(ix, queries, nq, k, L, nullptr, nullptr, false, params, out_ids, out_dist,
                       stream);
}

int bang_search_batched(bang_index *ix, const void *queries, uint32_t nq, const uint32_t *k_per_q,
                        const uint32_t *L_per_q, uint32_t k_max, uint32_t L_max,
                        const bang_search_params *params, uint32_t *out_ids, float *out_dist,
                        void *stream)
{
    return search_impl(ix, queries, nq, k_max, L_max, k_per_q, L_per_q, true, params, out_ids,
                       out_dist, stream);
}

int bang_pq_tables(bang_index *ix, const void *queries, uint32_t nq, void *out, uint32_t out_bf16,
                   void *stream)
{
    if (!ix || !queries || !out) return fail(BANG_EINVAL, "bang_pq_tables: NULL argument");
    if (!ix->have_pq) return fail(BANG_ESTATE, "bang_pq_tables: load the PQ data first");
    if (ix->dtype < 0) return fail(BANG_ESTATE, "bang_pq_tables: register the vectors first (element type)");
    if (!ix->tc_ok) return fail(BANG_EINVAL, "bang_pq_tables: unavailable for this PQ layout");
    if (!is_device_accessible(queries, ix->device) || !is_device_accessible(out, ix->device))
        return fail(BANG_EINVAL, "bang_pq_tables: queries and out must be device memory of the "
                    "index's device %d", ix->device);
    if (nq == 0) return BANG_OK;
    DeviceGuard g(ix->device);
    if (!g.ok) return fail(BANG_ECUDA, "cannot select device %d", ix->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bang::TcTableArgs ta;
    ta.queries = queries;
    ta.nq = nq; ta.d = ix->d; ta.M = ix->M;
    ta.off = ix->off;
    ta.btiles = static_cast<const unsigned char *>((out_bf16 & 2u) ? ix->tc_btiles_tf32.p : ix->tc_btiles.p);
    ta.bfirst = static_cast<const uint32_t *>(ix->tc_bfirst.p);
    ta.cnorm = static_cast<const float *>(ix->tc_cnorm.p);
    ta.out = out;
    ta.out_bf16 = (out_bf16 & 1u) ? 1u : 0u;
    ta.tf32 = (out_bf16 & 2u) ? 1u : 0u;
    ta.err = static_cast<unsigned int *>(ix->tc_err.p);
    CUDA_TRY(cudaMemsetAsync(ix->tc_err.p, 0, 4, st));
    cudaError_t te = bang::launch_tc_tables(ta, ix->dtype, st);
    if (te != cudaSuccess) return fail(BANG_ECUDA, "table kernel launch failed: %s", cudaGetErrorString(te));
    unsigned int flag = 0;
    CUDA_TRY(cudaMemcpyAsync(&flag, ix->tc_err.p, 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (flag) return fail(BANG_ETIMEOUT, "bang_pq_tables: a tensor-core wait gave up");
    return BANG_OK;
}

int bang_index_info(const bang_index *ix, uint64_t *n, uint32_t *d, uint32_t *M, uint32_t *R,
                    int32_t *dtype)
{
    if (!ix) return fail(BANG_EINVAL, "bang_index_info: index is NULL");
    if (n) *n = ix->n;
    if (d) *d = ix->d;
    if (M) *M = ix->M;
    if (R) *R = ix->R;
    if (dtype) *dtype = ix->dtype;
    return BANG_OK;
}

int bang_set_placement(bang_index *ix, uint32_t flags)
{
    if (!ix) return fail(BANG_EINVAL, "bang_set_placement: index is NULL");
    if (flags & ~(uint32_t)(BANG_GRAPH_IN_HBM | BANG_VECTORS_IN_HBM | BANG_GRAPH_PACKED | BANG_NEIGHBOR_CODES |
                            BANG_NODE_RECORDS))
        return fail(BANG_EINVAL, "bang_set_placement: unknown flags 0x%x", flags);
    if ((flags & BANG_NODE_RECORDS) && (flags & (BANG_GRAPH_IN_HBM | BANG_VECTORS_IN_HBM)))
        return fail(BANG_EINVAL, "bang_set_placement: node records are host memory; not with "
                    "BANG_GRAPH_IN_HBM or BANG_VECTORS_IN_HBM");
    if ((flags & BANG_NODE_RECORDS) && !(ix->have_graph && ix->have_vectors))
        return fail(BANG_ESTATE, "bang_set_placement: register the graph and the vectors first");
    if ((flags & BANG_NEIGHBOR_CODES) && (ix->R > 64 || ix->d > 128 || ix->Mpad > 32))
        return fail(BANG_EINVAL, "bang_set_placement: the neighbour-code layout needs R <= 64, d <= 128 "
                    "and M <= 32");
    if ((flags & (BANG_GRAPH_IN_HBM | BANG_GRAPH_PACKED | BANG_NEIGHBOR_CODES)) && !ix->have_graph)
        return fail(BANG_ESTATE, "bang_set_placement: register the graph first");
    if ((flags & BANG_VECTORS_IN_HBM) && !ix->have_vectors)
        return fail(BANG_ESTATE, "bang_set_placement: register the vectors first");
    DeviceGuard g(ix->device);
    if (!g.ok) return fail(BANG_ECUDA, "cannot select device %d", ix->device);
    CUDA_TRY(cudaDeviceSynchronize());
    if (flags & BANG_GRAPH_PACKED) {
        const int rc = build_packed_rows(ix);
        if (rc) return rc;
    }
    if ((flags & BANG_NEIGHBOR_CODES) && !ix->ncodes_ok) {
        CUDA_TRY(ix->ncodes.ensure((size_t)ix->n * ix->R * 32u));
        gather_neighbor_codes<<<1024, 256>>>(static_cast<const uint32_t *>(ix->adj.dev), ix->n, ix->R,
                                             ix->codes, ix->Mpad, static_cast<uint4 *>(ix->ncodes.p));
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaDeviceSynchronize());
        ix->ncodes_ok = true;
    } else if (!(flags & BANG_NEIGHBOR_CODES)) {
        ix->ncodes.release();
        ix->ncodes_ok = false;
    }
    if (flags & BANG_GRAPH_IN_HBM) {
        const bool pk = (flags & BANG_GRAPH_PACKED) != 0;
        const size_t bytes = (size_t)ix->n * (pk ? ix->adj_row_words : ix->R) * sizeof(uint32_t);
        ix->adj_hbm.release();
        CUDA_TRY(ix->adj_hbm.ensure(bytes));
        CUDA_TRY(cudaMemcpy(ix->adj_hbm.p, pk ? ix->adj_packed.host : ix->adj.host, bytes,
                            cudaMemcpyHostToDevice));
    } else {
        ix->adj_hbm.release();
    }
    if (flags & BANG_VECTORS_IN_HBM) {
        const size_t bytes = (size_t)ix->n * ix->d * elem_size(ix->dtype);
        CUDA_TRY(ix->base_hbm.ensure(bytes));
        CUDA_TRY(cudaMemcpy(ix->base_hbm.p, ix->base.host, bytes, cudaMemcpyHostToDevice));
    } else {
        ix->base_hbm.release();
    }
    if (flags & BANG_NODE_RECORDS) {
        const int rc = build_records(ix, (flags & BANG_GRAPH_PACKED) != 0);
        if (rc) return rc;
    } else {
        ix->records.release();
    }
    ix->placement = flags;
    return BANG_OK;
}

namespace {
struct HostBlock {
    void *raw;
    size_t bytes;
};
std::mutex g_host_mu;
std::map<void *, HostBlock> g_host_blocks;     // aligned address -> the whole mapping

// The transparent-huge-page size (2 MB on 4 KB-page systems, 512 MB on
// 64 KB-page arm64), or 2 MB when the system does not say.
size_t thp_size()
{
    size_t sz = 2u << 20;
    if (FILE *f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
        unsigned long long v = 0;
        if (std::fscanf(f, "%llu", &v) == 1 && v >= 4096 && (v & (v - 1)) == 0) sz = static_cast<size_t>(v);
        std::fclose(f);
    }
    return sz;
}
}  // namespace

int bang_host_alloc(uint64_t bytes, void **out)
{
    if (!out || bytes == 0) return fail(BANG_EINVAL, "bang_host_alloc: NULL output or zero bytes");
    *out = nullptr;
    const size_t align = thp_size();
    const size_t total = static_cast<size_t>(bytes) + align;
    void *raw = mmap(nullptr, total, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (raw == MAP_FAILED) return fail(BANG_ENOMEM, "bang_host_alloc: mmap of %zu bytes failed", total);
    const uintptr_t a = (reinterpret_cast<uintptr_t>(raw) + align - 1) & ~static_cast<uintptr_t>(align - 1);
    void *p = reinterpret_cast<void *>(a);
#ifdef MADV_HUGEPAGE
    madvise(p, static_cast<size_t>(bytes), MADV_HUGEPAGE);     // a hint: refused means 4 KB pages
#endif
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        g_host_blocks[p] = HostBlock{raw, total};
    }
    *out = p;
    return BANG_OK;
}

int bang_host_free(void *p)
{
    if (!p) return BANG_OK;
    HostBlock b;
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        auto it = g_host_blocks.find(p);
        if (it == g_host_blocks.end()) return fail(BANG_EINVAL, "bang_host_free: not from bang_host_alloc");
        b = it->second;
        g_host_blocks.erase(it);
    }
    munmap(b.raw, b.bytes);
    return BANG_OK;
}

int bang_destroy(bang_index *ix)
{
    if (!ix) return BANG_OK;
    {
        DeviceGuard g(ix->device);
        if (ix->codebook) cudaFree(ix->codebook);
        if (ix->off) cudaFree(ix->off);
        if (ix->codes) cudaFree(ix->codes);
        ix->adj.release();
        ix->adj_packed.release();
        ix->records.release();
        ix->ncodes.release();
        ix->base.release();
        ix->staging.release();
        ix->adj_hbm.release();
        ix->base_hbm.release();
        for (auto &kv : ix->work) kv.second.release();
        for (auto &kv : ix->tables) kv.second.release();
        for (auto &kv : ix->cands) kv.second.release();
        ix->tc_btiles.release();
        ix->tc_btiles_tf32.release();
        ix->tc_bfirst.release();
        ix->tc_cnorm.release();
        ix->tc_err.release();
    }
    delete ix;
    return BANG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free batched search.
//
// Some callers cannot let a library call cudaMalloc: a serving loop that must
// not stall on the implicit device-wide synchronisation cudaMalloc/cudaFree
// can cause, code recorded into a CUDA graph under global stream capture
// (where allocation calls are refused), or a host framework that owns the
// whole device-memory budget through its own pool.  For them the batched
// search has a variant whose scratch -- the work counter of the persistent
// launch, the per-L bucket cursors and the longest-L-first query order --
// lives in the file-scope array below instead of memory allocated per index
// and stream.  Every GPU that loads this library keeps the array
// (kNoAllocScratchWords * 4 bytes, about 270 KB) until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr uint32_t kNoAllocMaxQueries = 65536;           // queries per call, at most
constexpr uint32_t kNoAllocBuckets = bang::kMaxL + 1;     // L = 1..kMaxL; 0 = out of range
constexpr uint32_t kNoAllocCursor = 64;                   // word offsets in the array
constexpr uint32_t kNoAllocOrder = kNoAllocCursor + 2048;
constexpr uint32_t kNoAllocScratchWords = kNoAllocOrder + kNoAllocMaxQueries;

static __device__ __align__(256) unsigned int g_noalloc_scratch[kNoAllocScratchWords];

// One CTA of 1024 threads: zero the work counter and write the queries'
// order by decreasing L (counting sort; order within one L is arbitrary, and
// out-of-range L values go last, where the search flags them).
__global__ void __launch_bounds__(1024) noalloc_order_by_L(const uint32_t *L_per_q, uint32_t nq)
{
    __shared__ unsigned int hist[kNoAllocBuckets];
    __shared__ unsigned int scan[1024];
    unsigned int *cursor = g_noalloc_scratch + kNoAllocCursor;
    unsigned int *order = g_noalloc_scratch + kNoAllocOrder;
    const uint32_t t = threadIdx.x;
    for (uint32_t b = t; b < kNoAllocBuckets; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (uint32_t q = t; q < nq; q += blockDim.x) {
        const uint32_t L = L_per_q[q];
        atomicAdd(&hist[(L >= 1 && L <= (uint32_t)bang::kMaxL) ? L : 0u], 1u);
    }
    __syncthreads();
    // rank buckets by decreasing L: thread t owns bucket kMaxL - t (t < kMaxL)
    const uint32_t mine = hist[bang::kMaxL - t];
    scan[t] = mine;
    __syncthreads();
    for (uint32_t off = 1; off < 1024; off <<= 1) {
        const uint32_t v = t >= off ? scan[t - off] : 0u;
        __syncthreads();
        scan[t] += v;
        __syncthreads();
    }
    cursor[bang::kMaxL - t] = scan[t] - mine;                 // exclusive start
    if (t == 0) {
        cursor[0] = scan[1023];                               // out-of-range L last
        g_noalloc_scratch[0] = 0u;                            // work counter
    }
    __syncthreads();
    for (uint32_t q = t; q < nq; q += blockDim.x) {
        const uint32_t L = L_per_q[q];
        const uint32_t b = (L >= 1 && L <= (uint32_t)bang::kMaxL) ? L : 0u;
        order[atomicAdd(&cursor[b], 1u)] = q;
    }
}

std::mutex g_noalloc_mu;
unsigned int *g_noalloc_addr[128] = {};                       // per device ordinal

}  // namespace

extern "C" {

int bang_search_batched_noalloc(bang_index *ix, const void *queries, uint32_t nq,
                                const uint32_t *k_per_q, const uint32_t *L_per_q, uint32_t k_max,
                                uint32_t L_max, const bang_search_params *params,
                                uint32_t *out_ids, float *out_dist, void *stream)
{
    if (!ix) return fail(BANG_EINVAL, "bang_search_batched_noalloc: index is NULL");
    if (!ix->have_pq || !ix->have_graph || !ix->have_vectors)
        return fail(BANG_ESTATE, "bang_search_batched_noalloc: PQ data, graph and vectors must all be set");
    if (k_max == 0 || k_max > (uint32_t)bang::kMaxK)
        return fail(BANG_EINVAL, "bang_search_batched_noalloc: k_max=%u outside 1..%d", k_max, bang::kMaxK);
    if (L_max < k_max || L_max > (uint32_t)bang::kMaxL)
        return fail(BANG_EINVAL, "bang_search_batched_noalloc: L_max=%u must satisfy k_max <= L_max <= %d",
                    L_max, bang::kMaxL);
    if (nq > kNoAllocMaxQueries)
        return fail(BANG_EINVAL, "bang_search_batched_noalloc: nq=%u exceeds the %u queries its static "
                    "scratch holds; split the batch or use bang_search_batched", nq, kNoAllocMaxQueries);
    if (nq == 0) return BANG_OK;
    bang_search_params p;
    std::memset(&p, 0, sizeof p);
    if (params) p = *params;
    const uint32_t log2z = p.bloom_log2 ? p.bloom_log2 : 16u;
    if (log2z < 10 || log2z > 20)
        return fail(BANG_EINVAL, "bang_search_batched_noalloc: bloom_log2=%u outside 10..20", log2z);
    if (p.mode > 3) return fail(BANG_EINVAL, "bang_search_batched_noalloc: unknown mode %u", p.mode);
    if (p.trace && p.trace_cap == 0) return fail(BANG_EINVAL, "bang_search_batched_noalloc: trace_cap is 0");
    const void *ptrs[10] = {queries, k_per_q, L_per_q, out_ids, out_dist, p.out_iters, p.out_status,
                            p.out_ndist, p.trace, p.out_phase_cycles};
    for (int i = 0; i < 10; ++i) {
        if (i < 5 && !ptrs[i]) return fail(BANG_EINVAL, "bang_search_batched_noalloc: NULL buffer");
        if (ptrs[i] && !is_device_accessible(ptrs[i], ix->device))
            return fail(BANG_EINVAL, "bang_search_batched_noalloc: every buffer must be device memory "
                        "of the index's device %d (host buffers would need staging allocations)",
                        ix->device);
    }
    if (p.table_source != 0 && !(p.table_source == 3 && p.mode == 0))
        return fail(BANG_EINVAL, "bang_search_batched_noalloc: table_source must be 0, or 3 with mode 0 "
                    "(tensor-core tables need scratch)");
    if (p.rerank != 0)
        return fail(BANG_EINVAL, "bang_search_batched_noalloc: rerank must be 0 (candidate lists need scratch)");
    if (p.smem_carveout > 100)
        return fail(BANG_EINVAL, "bang_search_batched_noalloc: smem_carveout %u above 100", p.smem_carveout);
    const bool lazy = p.table_source == 3;
    const uint32_t ntab = lazy ? std::min(p.table_subspaces, ix->M) : 0u;
    bang::SmemLayout lay(ix->M, log2z, L_max, k_max, ix->d, ix->R, lazy ? (int)bang::kModeF32Lazy : (int)p.mode,
                         ntab);
    if (lay.total > 227u * 1024u)
        return fail(BANG_EINVAL, "bang_search_batched_noalloc: %u bytes of shared memory per query "
                    "exceed 227 KB", lay.total);

    DeviceGuard g(ix->device);
    if (!g.ok) return fail(BANG_ECUDA, "cannot select device %d", ix->device);
    unsigned int *scratch = nullptr;
    {
        // set-up, once per device, with that device current: the array's
        // device address (its name in host code is only a host-side stand-in)
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (ix->device < 0 || ix->device >= 128)
            return fail(BANG_EINVAL, "bang_search_batched_noalloc: device %d out of range", ix->device);
        if (!g_noalloc_addr[ix->device]) {
            void *addr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
            if (e != cudaSuccess)
                return fail(BANG_ECUDA, "bang_search_batched_noalloc: cudaGetSymbolAddress failed: %s",
                            cudaGetErrorString(e));
            g_noalloc_addr[ix->device] = static_cast<unsigned int *>(addr);
        }
        scratch = g_noalloc_addr[ix->device];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    noalloc_order_by_L<<<1, 1024, 0, st>>>(L_per_q, nq);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(BANG_ECUDA, "bang_search_batched_noalloc: order kernel launch failed: %s",
                    cudaGetErrorString(e));

    bang::SearchArgs a;
    std::memset(&a, 0, sizeof a);
    a.queries = queries;
    a.codebook = ix->codebook;
    a.off = ix->off;
    a.codes = ix->codes;
    set_graph_args(ix, a);
    a.n = (uint32_t)ix->n; a.d = ix->d; a.M = ix->M; a.Mpad = ix->Mpad; a.R = ix->R;
    a.medoid = ix->medoid;
    a.nq = nq; a.k = k_max; a.L = L_max; a.log2z = log2z; a.iter_cap = p.iter_cap;
    a.out_ids = out_ids;
    a.out_dist = out_dist;
    a.out_iters = p.out_iters;
    a.out_status = p.out_status;
    a.out_ndist = p.out_ndist;
    a.trace = p.trace;
    a.trace_cap = p.trace_cap;
    a.phase_cycles = p.out_phase_cycles;
    a.k_per_q = k_per_q;
    a.L_per_q = L_per_q;
    a.order = scratch + kNoAllocOrder;
    a.queue = scratch;
    a.grid_mult = p.grid_mult;
    a.spec = p.prefetch_depth >= 2 ? 1u : 0u;
    a.early_codes = p.early_codes ? 1u : 0u;
    a.carveout = p.smem_carveout;
    a.ntab = ntab;
    const uintptr_t qa = reinterpret_cast<uintptr_t>(a.queries);
    const uintptr_t ba = reinterpret_cast<uintptr_t>(a.base);
    a.vec_ok = (ix->d % 4 == 0) && (qa % 16 == 0) ? 1u : 0u;
    a.vecb_ok = (ix->d % 4 == 0) && (ba % 16 == 0) ? 1u : 0u;
    if (lazy) e = bang::launch_search_f32lazy(a, ix->dtype, lay.total, st);
    else if (p.mode == 0) e = bang::launch_search_f32(a, ix->dtype, lay.total, st);
    else if (p.mode == 1) e = bang::launch_search_bf16(a, ix->dtype, lay.total, st);
    else if (p.mode == 3) e = bang::launch_search_q8(a, ix->dtype, lay.total, st);
    else e = bang::launch_search_exact(a, ix->dtype, lay.total, st);
    if (e != cudaSuccess)
        return fail(BANG_ECUDA, "bang_search_batched_noalloc: search kernel launch failed: %s",
                    cudaGetErrorString(e));
    return BANG_OK;
}

}  // extern "C"
