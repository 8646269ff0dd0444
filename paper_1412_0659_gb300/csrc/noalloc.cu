// noalloc.cu -- bonsai_sfc_order_noalloc: the bounding cube, Peano-Hilbert
// keys and their stable sort for callers that may not allocate device
// memory (see include/bonsai_gb.h for who they are).  The kernels are the
// library's own key and sort kernels; only their scratch differs: it lives
// in one file-scope static device array instead of context allocations.
#include <mutex>

#include "internal.cuh"

namespace {

using bgb::BoxPartial;
using bgb::DevScalars;

constexpr int64_t MAX_N = BONSAI_NOALLOC_MAX_N;
constexpr int MAX_PART = 1024;  // bounding-box block partials
constexpr int MAX_DEVICES = 64;

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// byte offsets of the regions of the scratch array
constexpr size_t OFF_KEY2 = 0;
constexpr size_t OFF_VAL2 = OFF_KEY2 + align256(sizeof(uint64_t) * MAX_N);
constexpr size_t SORT_ELEMS = bgb::sort_scratch_elems(MAX_N);
constexpr size_t OFF_SORT = OFF_VAL2 + align256(sizeof(uint32_t) * MAX_N);
constexpr size_t OFF_PART = OFF_SORT + align256(sizeof(uint32_t) * SORT_ELEMS);
constexpr size_t OFF_DSC = OFF_PART + align256(sizeof(BoxPartial) * MAX_PART);
constexpr size_t SCRATCH_BYTES = OFF_DSC + align256(sizeof(DevScalars));
// the sort's region is sized from its own tile constants, so a retuned sort
// cannot write past it; the total stays modest
static_assert(OFF_PART - OFF_SORT >= sizeof(uint32_t) * bgb::sort_scratch_elems(MAX_N), "sort region");
static_assert(OFF_SORT % 8 == 0, "the sort's descriptors are 64-bit words");
static_assert(SCRATCH_BYTES < (16u << 20), "scratch array above 16 MB");

// The scratch of every call on this device.  Host code must not use its name
// as an address: the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

std::mutex g_mu;
unsigned char *g_base[MAX_DEVICES] = {};
int g_sms[MAX_DEVICES] = {};

// Once per device, with that device current: the device address of the
// scratch array and the SM count.
int setup(int dev, unsigned char **base, int *sms) {
    if (dev < 0 || dev >= MAX_DEVICES) return BONSAI_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return BONSAI_ECUDA;
        }
        int s = 0;
        if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s < 1)
            return BONSAI_ECUDA;
        g_sms[dev] = s;
        g_base[dev] = static_cast<unsigned char *>(p);
    }
    *base = g_base[dev];
    *sms = g_sms[dev];
    return BONSAI_OK;
}

}  // namespace

extern "C" int bonsai_sfc_order_noalloc(const double *pos, const double *mass, int64_t n,
                                        uint64_t *keys, uint32_t *perm, double cube[4],
                                        void *stream) {
    if (!pos || !mass || !keys || !perm || n < 1 || n > MAX_N) return BONSAI_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return BONSAI_ECUDA;
    unsigned char *base = nullptr;
    int sms = 0;
    int rc = setup(dev, &base, &sms);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t *key2 = reinterpret_cast<uint64_t *>(base + OFF_KEY2);
    uint32_t *val2 = reinterpret_cast<uint32_t *>(base + OFF_VAL2);
    uint32_t *sort_scratch = reinterpret_cast<uint32_t *>(base + OFF_SORT);
    BoxPartial *part = reinterpret_cast<BoxPartial *>(base + OFF_PART);
    DevScalars *dsc = reinterpret_cast<DevScalars *>(base + OFF_DSC);
    // the status word and cube of the previous call are still there: clear them
    BGB_CUDA(cudaMemsetAsync(dsc, 0, sizeof(DevScalars), s));
    bgb::launch_cube_keys_into(s, sms, pos, mass, n, part, MAX_PART, dsc, keys, perm);
    // eight passes ping-pong between the caller's buffers and the scratch halves
    bgb::radix_sort_pairs_into(s, sms, n, keys, key2, perm, val2, sort_scratch, &dsc->status);
    BGB_CUDA(cudaGetLastError());
    DevScalars h;
    BGB_CUDA(cudaMemcpyAsync(&h, dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    BGB_WAIT(s);
    if (h.status & bgb::ST_BAD_INPUT) return BONSAI_EINVAL;
    if (h.status & bgb::ST_TIMEOUT) return BONSAI_ETIMEOUT;
    if (cube) {
        cube[0] = h.lo[0];
        cube[1] = h.lo[1];
        cube[2] = h.lo[2];
        cube[3] = h.L;
    }
    return BONSAI_OK;
}
