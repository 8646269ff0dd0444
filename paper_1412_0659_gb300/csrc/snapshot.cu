// snapshot.cu -- snapshots of the FP64 state for restarting and for
// analysis, and the face-on surface density computed on the fly (Sec. VI.C:
// intermediate snapshots are stored "for the dual purpose of restarting and
// detailed analysis", next to rudimentary on-the-fly analysis; Sec. IV,
// Fig. 4: the face-on surface density of the disk and the bulge).
//
// File format (little-endian): a 64-byte header {"BONSAIGB", version 1,
// flags 0, n, time, G, theta, eps, 2 reserved words}, then pos [3][n],
// vel [3][n] and mass [n] as float64 in caller order.  Transfers stream
// through two pinned staging buffers: the device copy of one chunk
// overlaps the file write (or read) of the other.
#include <stdio.h>
#include <string.h>

#include "internal.cuh"

namespace bgb {

namespace {

struct SnapshotHeader {
    char magic[8];
    uint32_t version;
    uint32_t flags;
    int64_t n;
    double time;
    double G;
    float theta, eps;
    uint64_t reserved[2];
};
static_assert(sizeof(SnapshotHeader) == 64, "snapshot header layout");

const char kMagic[8] = {'B', 'O', 'N', 'S', 'A', 'I', 'G', 'B'};
constexpr size_t STAGE_BYTES = size_t(64) << 20;

int ensure_stage(bonsai_ctx *c) {
    for (int k = 0; k < 2; ++k) {
        if (c->stage[k]) continue;
        if (cudaMallocHost(&c->stage[k], STAGE_BYTES) != cudaSuccess) {
            cudaGetLastError();
            c->stage[k] = nullptr;
            return BONSAI_ENOMEM;
        }
    }
    return BONSAI_OK;
}

struct Span {
    char *dev;
    size_t bytes;
};

// The three arrays cut into chunks of at most STAGE_BYTES.
int chunks(bonsai_ctx *c, Span out[], int cap, double *pos, double *vel, double *mass) {
    const size_t n = (size_t)c->n;
    const Span whole[3] = {{reinterpret_cast<char *>(pos), 3 * n * sizeof(double)},
                           {reinterpret_cast<char *>(vel), 3 * n * sizeof(double)},
                           {reinterpret_cast<char *>(mass), n * sizeof(double)}};
    int k = 0;
    for (const Span &w : whole)
        for (size_t o = 0; o < w.bytes; o += STAGE_BYTES) {
            if (k == cap) return -1;
            out[k++] = Span{w.dev + o, w.bytes - o < STAGE_BYTES ? w.bytes - o : STAGE_BYTES};
        }
    return k;
}

constexpr int MAX_CHUNKS = 4096;  // 256 GB of state

// Face-on (x-y) cloud-in-cell surface density of the particles whose caller
// index is in [first, first + count): each deposits m / (hx hy) with bilinear
// weights onto the four nearest pixel centres; pixels outside are dropped.
__global__ void __launch_bounds__(256) k_surface_density(
    const double *__restrict__ pos, const double *__restrict__ mass,
    const uint32_t *__restrict__ id, int64_t n, uint32_t first, uint32_t count, double x0,
    double y0, double hx, double hy, int nx, int ny, double *__restrict__ map) {
    const double inv_area = 1.0 / (hx * hy);
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        if (id[i] - first >= count) continue;
        const double fx = (pos[i] - x0) / hx - 0.5;
        const double fy = (pos[n + i] - y0) / hy - 0.5;
        if (!(fx > -1.0 && fx < (double)nx && fy > -1.0 && fy < (double)ny)) continue;
        const double ix = floor(fx), iy = floor(fy);
        const double tx = fx - ix, ty = fy - iy;
        const int jx = (int)ix, jy = (int)iy;
        const double w = mass[i] * inv_area;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int px = jx + dx, py = jy + dy;
                if (px < 0 || px >= nx || py < 0 || py >= ny) continue;
                const double wx = dx ? tx : 1.0 - tx, wy = dy ? ty : 1.0 - ty;
                atomicAdd(&map[(int64_t)py * nx + px], w * wx * wy);
            }
    }
}

}  // namespace

}  // namespace bgb

using namespace bgb;

extern "C" int tree_save_snapshot(bonsai_ctx *c, const char *path, double time) {
    if (!c || !path) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    int rc = ensure_stage(c);
    if (rc) return rc;
    // caller-order copies in the second halves of the state buffers, which
    // are free between steps
    launch_unpermute_state(c, c->pos2.p, c->vel2.p, c->mass2.p);
    Span ch[MAX_CHUNKS];
    const int nch = chunks(c, ch, MAX_CHUNKS, c->pos2.p, c->vel2.p, c->mass2.p);
    if (nch < 0) return BONSAI_EINVAL;
    FILE *f = fopen(path, "wb");
    if (!f) return BONSAI_EIO;
    SnapshotHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kMagic, 8);
    h.version = 1;
    h.n = c->n;
    h.time = time;
    h.G = c->prm.G;
    h.theta = c->prm.theta;
    h.eps = c->prm.eps;
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1;
    cudaEvent_t ev[2] = {c->ev[0], c->ev[1]};
    for (int k = 0; k <= nch && ok; ++k) {
        if (k < nch) {
            if (cudaMemcpyAsync(c->stage[k & 1], ch[k].dev, ch[k].bytes, cudaMemcpyDeviceToHost,
                                c->stream) != cudaSuccess ||
                cudaEventRecord(ev[k & 1], c->stream) != cudaSuccess) {
                ok = false;
                break;
            }
        }
        if (k > 0) {  // write the previous chunk while this one copies
            const int p = (k - 1) & 1;
            if (cudaEventSynchronize(ev[p]) != cudaSuccess) {
                ok = false;
                break;
            }
            ok = fwrite(c->stage[p], 1, ch[k - 1].bytes, f) == ch[k - 1].bytes;
        }
    }
    if (fclose(f) != 0) ok = false;
    if (!ok) {
        const int w = wait_stream(c->stream);
        if (w != BONSAI_OK) return w;
        return cudaGetLastError() != cudaSuccess ? BONSAI_ECUDA : BONSAI_EIO;
    }
    return BONSAI_OK;
}

extern "C" int tree_load_snapshot(bonsai_ctx *c, const char *path, double *time) {
    if (!c || !path) return BONSAI_EINVAL;
    FILE *f = fopen(path, "rb");
    if (!f) return BONSAI_EIO;
    SnapshotHeader h;
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, kMagic, 8) != 0 || h.version != 1 ||
        h.n < 1 || h.n > 0x7fffffffll) {
        fclose(f);
        return BONSAI_EIO;
    }
    // the file must hold exactly the header and 7 n doubles
    const long long want = (long long)sizeof(h) + 7ll * 8ll * h.n;
    if (fseeko(f, 0, SEEK_END) != 0 || (long long)ftello(f) != want ||
        fseeko(f, (off_t)sizeof(h), SEEK_SET) != 0) {
        fclose(f);
        return BONSAI_EIO;
    }
    c->have_tree = c->have_forces = c->have_vel = false;
    c->n = h.n;
    int rc = particle_buffers(c, h.n);
    if (!rc) rc = ensure_stage(c);
    if (rc) {
        fclose(f);
        return rc;
    }
    Span ch[MAX_CHUNKS];
    const int nch = chunks(c, ch, MAX_CHUNKS, c->pos2.p, c->vel2.p, c->mass2.p);
    bool ok = nch >= 0;
    cudaEvent_t ev[2] = {c->ev[0], c->ev[1]};
    for (int k = 0; k < nch && ok; ++k) {
        const int b = k & 1;
        if (k >= 2 && cudaEventSynchronize(ev[b]) != cudaSuccess) {  // staging half free again
            ok = false;
            break;
        }
        ok = fread(c->stage[b], 1, ch[k].bytes, f) == ch[k].bytes;  // overlaps the copy of k-1
        if (ok)
            ok = cudaMemcpyAsync(ch[k].dev, c->stage[b], ch[k].bytes, cudaMemcpyHostToDevice,
                                 c->stream) == cudaSuccess &&
                 cudaEventRecord(ev[b], c->stream) == cudaSuccess;
    }
    fclose(f);
    BGB_WAIT(c->stream);
    if (!ok) return BONSAI_EIO;
    rc = rebuild(c, c->pos2.p, c->mass2.p, true);
    if (rc) return rc;
    c->stats.n = c->n;
    c->stats.n_nodes = c->n_nodes;
    c->stats.n_groups = c->n_groups;
    c->stats.depth = c->depth;
    launch_permute_in_vel(c, c->vel2.p);
    BGB_WAIT(c->stream);
    c->have_vel = true;
    if (time) *time = h.time;
    return BONSAI_OK;
}

extern "C" int tree_surface_density(bonsai_ctx *c, int64_t first, int64_t count,
                                    const double window[4], int nx, int ny, double *map) {
    if (!c || !window || !map || nx < 1 || ny < 1 || first < 0 || count < 0) return BONSAI_EINVAL;
    if (!(window[1] > window[0]) || !(window[3] > window[2]) || !isfinite(window[0]) ||
        !isfinite(window[1]) || !isfinite(window[2]) || !isfinite(window[3]))
        return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    if (first > c->n || count > c->n - first) return BONSAI_EINVAL;
    const double hx = (window[1] - window[0]) / nx, hy = (window[3] - window[2]) / ny;
    BGB_CUDA(cudaMemsetAsync(map, 0, sizeof(double) * (size_t)nx * (size_t)ny, c->stream));
    k_surface_density<<<grid_for(c->n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        c->pos.p, c->mass.p, c->id.p, c->n, (uint32_t)first, (uint32_t)count, window[0],
        window[2], hx, hy, nx, ny, map);
    c->launches += 1;
    BGB_CUDA(cudaPeekAtLastError());
    BGB_WAIT(c->stream);
    return BONSAI_OK;
}
