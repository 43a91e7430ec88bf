// checkpoint.cu - save and restore a grid's state to and from a file
// (mrt_save / mrt_load; the paper has no counterpart).
//
// File layout (little-endian, as both host architectures are):
//   CkptHeader (below), then the current distribution buffer in the padded
//   device layout, 16 * plane elements of the grid precision: the data, the
//   ghost columns and rows (fixed-equilibrium ghosts included, so a resumed
//   run needs no knowledge of the initial fields) and the padding.
// The payload checksum is FNV-1a over its 64-bit words (a trailing partial
// word, which the layout never has, would be ignored).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "host_state.h"

using namespace mrt;

namespace {

constexpr char kMagic[8] = {'M', 'R', 'T', 'F', 'D', 'L', 'B', '1'};
constexpr unsigned kVersion = 1;

struct CkptHeader {
    char magic[8];
    unsigned version;
    int nx, ny, precision, advection, bc_x, bc_y, G;
    long pitch, plane, steps;
    double dx, dt, gamma, s[16];   // s after the Pr rule (as stepped)
    unsigned long long checksum;   // FNV-1a over the payload's 64-bit words
    unsigned long long payload_bytes;
};

unsigned long long fnv1a64(const void* data, size_t bytes) {
    const unsigned long long* w = static_cast<const unsigned long long*>(data);
    unsigned long long h = 1469598103934665603ull;
    for (size_t k = 0; k < bytes / 8; ++k) {
        h ^= w[k];
        h *= 1099511628211ull;
    }
    return h;
}

void fill_header(const mrt_grid* g, CkptHeader* h, size_t payload) {
    std::memset(h, 0, sizeof *h);
    std::memcpy(h->magic, kMagic, 8);
    h->version = kVersion;
    h->nx = g->L.nx;
    h->ny = g->L.ny;
    h->precision = g->p.precision;
    h->advection = g->p.advection;
    h->bc_x = g->p.bc_x;
    h->bc_y = g->p.bc_y;
    h->G = g->L.G;
    h->pitch = g->L.pitch;
    h->plane = g->L.plane;
    h->steps = g->steps;
    h->dx = g->p.dx;
    h->dt = g->p.dt;
    h->gamma = g->p.gamma;
    for (int k = 0; k < 16; ++k) h->s[k] = g->p.s[k];
    h->payload_bytes = payload;
}

}  // namespace

extern "C" mrt_status mrt_save(mrt_grid* g, const char* path) {
    NvtxRange range("mrt_save");
    if (!g || !path) return mrt_fail(MRT_EINVAL, "null argument");
    const size_t bytes = 16 * (size_t)g->L.plane * g->elem;
    std::vector<unsigned char> host;
    try {
        host.resize(bytes);
    } catch (...) {
        return mrt_fail(MRT_ENOMEM, "host buffer of %zu bytes", bytes);
    }
    cudaError_t e = cudaMemcpyAsync(host.data(), g->f[g->cur], bytes, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "state copy: %s", cudaGetErrorString(e));
    CkptHeader h;
    fill_header(g, &h, bytes);
    h.checksum = fnv1a64(host.data(), bytes);
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return mrt_fail(MRT_EINVAL, "cannot open %s for writing", path);
    const bool ok = std::fwrite(&h, sizeof h, 1, fp) == 1 && std::fwrite(host.data(), 1, bytes, fp) == bytes;
    const bool closed = std::fclose(fp) == 0;
    if (!ok || !closed) return mrt_fail(MRT_EINVAL, "short write to %s", path);
    return MRT_OK;
}

extern "C" mrt_status mrt_load(mrt_grid* g, const char* path) {
    NvtxRange range("mrt_load");
    if (!g || !path) return mrt_fail(MRT_EINVAL, "null argument");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return mrt_fail(MRT_EINVAL, "cannot open %s", path);
    CkptHeader h;
    if (std::fread(&h, sizeof h, 1, fp) != 1 || std::memcmp(h.magic, kMagic, 8) != 0) {
        std::fclose(fp);
        return mrt_fail(MRT_EINVAL, "%s is not a checkpoint of this library", path);
    }
    if (h.version != kVersion) {
        std::fclose(fp);
        return mrt_fail(MRT_EINVAL, "checkpoint version %u, expected %u", h.version, kVersion);
    }
    CkptHeader want;
    const size_t bytes = 16 * (size_t)g->L.plane * g->elem;
    fill_header(g, &want, bytes);
    const char* diff = nullptr;
    if (h.nx != want.nx || h.ny != want.ny) diff = "grid size";
    else if (h.precision != want.precision) diff = "precision";
    else if (h.advection != want.advection) diff = "advection operator";
    else if (h.bc_x != want.bc_x || h.bc_y != want.bc_y) diff = "boundary kinds";
    else if (h.G != want.G || h.pitch != want.pitch || h.plane != want.plane || h.payload_bytes != bytes)
        diff = "padded layout";
    else if (h.dx != want.dx || h.dt != want.dt || h.gamma != want.gamma ||
             std::memcmp(h.s, want.s, sizeof h.s) != 0)
        diff = "dx, dt, gamma or relaxation rates";
    if (diff) {
        std::fclose(fp);
        return mrt_fail(MRT_EINVAL, "checkpoint %s does not match the grid's %s", path, diff);
    }
    std::vector<unsigned char> host;
    try {
        host.resize(bytes);
    } catch (...) {
        std::fclose(fp);
        return mrt_fail(MRT_ENOMEM, "host buffer of %zu bytes", bytes);
    }
    const bool ok = std::fread(host.data(), 1, bytes, fp) == bytes;
    std::fclose(fp);
    if (!ok) return mrt_fail(MRT_EINVAL, "checkpoint %s is truncated", path);
    if (fnv1a64(host.data(), bytes) != h.checksum) return mrt_fail(MRT_EINVAL, "checkpoint %s: checksum mismatch", path);
    // both buffers: the fixed ghosts live in both; the other buffer's data is
    // rewritten by the next step
    for (int b = 0; b < 2; ++b) {
        cudaError_t e = cudaMemcpyAsync(g->f[b], host.data(), bytes, cudaMemcpyHostToDevice, g->stream);
        if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "state copy: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return mrt_fail(MRT_ECUDA, "state copy: %s", cudaGetErrorString(e));
    g->steps = h.steps;
    g->totals_fresh = false;
    return MRT_OK;
}
