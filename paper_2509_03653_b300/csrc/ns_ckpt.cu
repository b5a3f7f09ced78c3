// ns_ckpt.cu -- checkpoint and resume of a traffic matrix.
//
// A checkpoint holds A's sorted nonzero list -- the paper's three-column
// frame (src, dst, n_packets; section "Implementation") -- and its nine
// Table 2 quantities.  Saving exports the list (sorted on the GPU) and
// writes it beside the target path, then renames it over the target.
// Loading checks the file, inserts the entries into an emptied matrix with
// the library's own insert kernels (so every quantity is recomputed on the
// GPU), and compares the recomputed quantities with the saved ones.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ns.h"
#include "ns_api_internal.h"

using namespace ns;

namespace {

constexpr char kMagic[8] = {'N', 'S', 'M', 'A', 'T', 'R', 'I', 'X'};
constexpr uint32_t kHeaderBytes = 128;

struct Header {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    uint64_t nnz;
    uint64_t stats[S_NFIELDS];
    uint64_t pad[(kHeaderBytes - 24 - 8 * S_NFIELDS) / 8];
};
static_assert(sizeof(Header) == kHeaderBytes, "checkpoint header is 128 bytes");

ns_status cuda_fail(const char* what, cudaError_t e) {
    cudaGetLastError();
    return fail_fmt(NS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool write_all(FILE* f, const void* p, size_t bytes) { return bytes == 0 || fwrite(p, 1, bytes, f) == bytes; }
bool read_all(FILE* f, void* p, size_t bytes) { return bytes == 0 || fread(p, 1, bytes, f) == bytes; }

}  // namespace

extern "C" {

ns_status ns_matrix_save(const ns_matrix* m, const char* path, ns_stream_t stream) {
    if (!m || !path) return set_fail(NS_ERR_INVALID, "ns_matrix_save: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    CallScope scope(m->ctx, s);
    touch(m, s);
    DevStats ds;
    ns_status st = read_stats(m, s, &ds);
    if (st != NS_OK) return st;
    const uint64_t nnz = ds.v[S_LINKS];
    std::vector<uint64_t> keys(nnz), counts(nnz);
    if (nnz) {
        Buf dk, dc;
        st = buf_reserve(dk, nnz * sizeof(uint64_t));
        if (st == NS_OK) st = buf_reserve(dc, nnz * sizeof(uint64_t));
        uint64_t got = 0;
        if (st == NS_OK) st = ns_matrix_export(m, (uint64_t*)dk.p, (uint64_t*)dc.p, nnz, &got, stream);
        if (st == NS_OK && got != nnz) st = set_fail(NS_ERR_STATE, "ns_matrix_save: the matrix changed while saved");
        // copies on the caller's stream, behind the export (a legacy-stream
        // cudaMemcpy is not ordered with a non-blocking stream)
        cudaError_t e = cudaSuccess;
        if (st == NS_OK)
            e = cudaMemcpyAsync(keys.data(), dk.p, nnz * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
        if (st == NS_OK && e == cudaSuccess)
            e = cudaMemcpyAsync(counts.data(), dc.p, nnz * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
        if (st == NS_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (st == NS_OK && e != cudaSuccess) st = cuda_fail("ns_matrix_save: copy to host", e);
        buf_free(dk);
        buf_free(dc);
        if (st != NS_OK) return st;
    }
    Header h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kMagic, sizeof kMagic);
    h.version = NS_CHECKPOINT_VERSION;
    h.header_bytes = kHeaderBytes;
    h.nnz = nnz;
    for (int i = 0; i < S_NFIELDS; ++i) h.stats[i] = ds.v[i];
    const std::string tmp = std::string(path) + ".partial";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return fail_fmt(NS_ERR_IO, "ns_matrix_save: cannot create %s", tmp.c_str());
    bool ok = write_all(f, &h, sizeof h) && write_all(f, keys.data(), nnz * sizeof(uint64_t)) &&
              write_all(f, counts.data(), nnz * sizeof(uint64_t));
    ok = (std::fflush(f) == 0) && ok;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return fail_fmt(NS_ERR_IO, "ns_matrix_save: cannot write %s", path);
    }
    return NS_OK;
}

ns_status ns_matrix_load(ns_ctx* c, const char* path, ns_matrix* m, ns_stream_t stream) {
    if (!c || !path || !m) return set_fail(NS_ERR_INVALID, "ns_matrix_load: NULL argument");
    if (m->ctx != c) return set_fail(NS_ERR_INVALID, "ns_matrix_load: matrix belongs to another context");
    cudaStream_t s = (cudaStream_t)stream;
    CallScope scope(c, s);
    touch(m, s);
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail_fmt(NS_ERR_IO, "ns_matrix_load: cannot open %s", path);
    Header h;
    bool ok = read_all(f, &h, sizeof h);
    long size = -1;
    if (ok && std::fseek(f, 0, SEEK_END) == 0) size = std::ftell(f);
    ns_status bad = NS_OK;
    if (!ok || std::memcmp(h.magic, kMagic, sizeof kMagic) != 0)
        bad = set_fail(NS_ERR_INVALID, "ns_matrix_load: not a matrix checkpoint");
    else if (h.version != NS_CHECKPOINT_VERSION || h.header_bytes != kHeaderBytes)
        bad = fail_fmt(NS_ERR_INVALID, "ns_matrix_load: unsupported checkpoint version %u", h.version);
    else if (size < 0 || h.nnz > ((uint64_t)size) / 16 ||
             (uint64_t)size != (uint64_t)kHeaderBytes + 16 * h.nnz)
        bad = set_fail(NS_ERR_INVALID, "ns_matrix_load: file size does not match its entry count");
    const uint64_t nnz = bad == NS_OK ? h.nnz : 0;
    std::vector<uint64_t> keys, counts;
    if (bad == NS_OK) {
        keys.resize(nnz);
        counts.resize(nnz);
        ok = std::fseek(f, (long)kHeaderBytes, SEEK_SET) == 0 && read_all(f, keys.data(), nnz * sizeof(uint64_t)) &&
             read_all(f, counts.data(), nnz * sizeof(uint64_t));
        if (!ok) bad = fail_fmt(NS_ERR_IO, "ns_matrix_load: cannot read %s", path);
    }
    std::fclose(f);
    if (bad != NS_OK) return bad;
    for (uint64_t i = 0; i < nnz; ++i) {
        if (counts[i] == 0 || (i > 0 && keys[i] <= keys[i - 1]))
            return set_fail(NS_ERR_INVALID, "ns_matrix_load: keys not strictly ascending, or a zero count");
    }
    // insert the entries into the emptied matrix as a sorted nonzero list
    ns_status st = ns_matrix_clear(m, stream);
    if (st != NS_OK) return st;
    if (nnz) {
        ns_matrix tmp;
        tmp.ctx = c;
        tmp.device = c->device;
        tmp.fmt = FMT_LIST;
        tmp.bound = nnz;
        DevStats ts;
        std::memset(&ts, 0, sizeof ts);
        ts.v[S_LINKS] = nnz;  // the list's length, which the insert kernel reads
        st = buf_reserve(tmp.keys, nnz * sizeof(uint64_t));
        if (st == NS_OK) st = buf_reserve(tmp.counts, nnz * sizeof(uint64_t));
        if (st == NS_OK) st = buf_reserve(tmp.stats, sizeof(DevStats));
        // The copies go on the caller's stream, ahead of the insert that
        // reads them: a pageable cudaMemcpy may return before its transfer
        // has landed, and the legacy stream it uses is not ordered with a
        // non-blocking one.  The host vectors outlive the synchronization
        // below.
        cudaError_t e = cudaSuccess;
        if (st == NS_OK)
            e = cudaMemcpyAsync(tmp.keys.p, keys.data(), nnz * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
        if (st == NS_OK && e == cudaSuccess)
            e = cudaMemcpyAsync(tmp.counts.p, counts.data(), nnz * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
        if (st == NS_OK && e == cudaSuccess) e = cudaMemcpyAsync(tmp.stats.p, &ts, sizeof ts, cudaMemcpyHostToDevice, s);
        if (st == NS_OK && e != cudaSuccess) st = cuda_fail("ns_matrix_load: copy to device", e);
        if (st == NS_OK) st = ns_accumulate(c, m, &tmp, stream);
        // the temporaries are freed only once the stream is past every
        // command that reads them, also when a step above failed
        const cudaError_t se = cudaStreamSynchronize(s);
        if (st == NS_OK && se != cudaSuccess) st = cuda_fail("ns_matrix_load: insert", se);
        buf_free(tmp.keys);
        buf_free(tmp.counts);
        buf_free(tmp.stats);
        if (st != NS_OK) {
            // never leave a partly loaded matrix behind
            ns_matrix_clear(m, stream);
            return st;
        }
    }
    DevStats got;
    st = read_stats(m, s, &got);
    if (st != NS_OK) {
        ns_matrix_clear(m, stream);
        return st;
    }
    for (int i = 0; i < S_NFIELDS; ++i) {
        if (got.v[i] != h.stats[i]) {
            ns_matrix_clear(m, stream);
            return fail_fmt(NS_ERR_INVALID, "ns_matrix_load: recomputed quantity %d is %llu, the file says %llu", i,
                            (unsigned long long)got.v[i], (unsigned long long)h.stats[i]);
        }
    }
    return NS_OK;
}

}  // extern "C"
