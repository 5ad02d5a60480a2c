// wilson_apply_noalloc: the Wilson-Dirac operator for callers that cannot allocate
// device memory.
//
// Some callers must not call cudaMalloc/cudaFree at all: a runtime that owns every
// byte of device memory through its own pool (a foreign allocation would bypass its
// budget and accounting), or a latency-critical service loop where cudaFree's implicit
// device-wide synchronisation would stall every other stream. Such callers also cannot
// create a context (ovl_create allocates its workspace). This entry point needs neither:
// its working memory is one file-scope device array of fixed size, reserved when the
// library is loaded and held by every GPU that loads it until the process exits.
//
// Working memory (FP64, even-odd layouts of the library): the links of all four
// directions, the packed input spinor and the packed output spinor, for at most
// kNoAllocMaxSites lattice sites (about 15.7 MB in total).
#include <mutex>
#include <string>

#include "../../include/ovl.h"
#include "internal.h"

namespace ovl {

constexpr long kNoAllocMaxSites = 16384;
constexpr size_t kNoAllocLinkBytes = (size_t)kNoAllocMaxSites * 4 * kLink64Words * sizeof(double2);
constexpr size_t kNoAllocSpinorBytes = (size_t)kNoAllocMaxSites * 12 * sizeof(double2);
constexpr size_t kNoAllocBytes = kNoAllocLinkBytes + 2 * kNoAllocSpinorBytes;

// The shared working memory. Every call overwrites all of the part it reads (links,
// input and output spinor for its V sites), so nothing has to start at zero.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

// Every link into the FP64 even-odd link layout of the library (all 18 reals of
// kLinkScale U, the form the stencil expects).
__global__ void k_noalloc_pack_links(Geom g, const double2 *__restrict__ lex) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)g.V * 4) return;
    const int s = (int)(t >> 2), mu = (int)(t & 3);
    int r = s;
    const int x3 = r % g.L[3]; r /= g.L[3];
    const int x2 = r % g.L[2]; r /= g.L[2];
    const int x1 = r % g.L[1];
    const int x0 = r / g.L[1];
    const int p = (x0 + x1 + x2 + x3) & 1, i = s >> 1;
    double2 *links = reinterpret_cast<double2 *>(g_noalloc_scratch);
    double2 *d = links + ((size_t)(p * 4 + mu) * kLink64Words) * g.Vh + i;
#pragma unroll
    for (int c = 0; c < 9; c++) {
        const double2 w = lex[(size_t)t * 9 + c];
        d[(size_t)c * g.Vh] = make_double2(kLinkScale * w.x, kLinkScale * w.y);
    }
}

std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
void *g_noalloc_addr[kMaxDevices] = {};   // device address of the array, per device

ovl_status fail(ovl_status s, const std::string &msg) {
    set_thread_error(msg);   // read back with ovl_last_error(NULL)
    return s;
}

// Device memory of device dev (or managed memory): a pointer into another GPU's memory is
// refused, since the kernels run on the current device.
bool device_ptr(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

}  // namespace

}  // namespace ovl

using namespace ovl;

extern "C" ovl_status wilson_apply_noalloc(double *out, const double *in, const double *gauge, const int dims[4],
                                           double m0, int antiperiodic, void *cuda_stream) {
    if (!out || !in || !gauge || !dims) return fail(OVL_EINVAL, "wilson_apply_noalloc: NULL argument");
    if (!isfinite(m0)) return fail(OVL_EINVAL, "wilson_apply_noalloc: m0 must be finite");
    long V = 1;
    for (int m = 0; m < 4; m++) {
        if (dims[m] < 2 || (dims[m] & 1))
            return fail(OVL_EINVAL, "wilson_apply_noalloc: lattice extents must be even and >= 2");
        V *= dims[m];
    }
    if (V > kNoAllocMaxSites)
        return fail(OVL_EINVAL, "wilson_apply_noalloc: lattice of " + std::to_string(V) +
                                    " sites exceeds the fixed working memory of " +
                                    std::to_string(kNoAllocMaxSites) + " sites");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail(OVL_ECUDA, "wilson_apply_noalloc: no usable current device");
    }
    if (!device_ptr(out, dev) || !device_ptr(in, dev) || !device_ptr(gauge, dev))
        return fail(OVL_EINVAL, "wilson_apply_noalloc: out, in and gauge must be memory of the current device");
    // Address of the working memory on the current device, looked up once per device and
    // kept for the life of the process (the primary context of that device; a
    // cudaDeviceReset or another driver context makes it stale, see include/ovl.h).
    unsigned char *scratch;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *addr = nullptr;
            e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
            if (e != cudaSuccess || !addr) {
                cudaGetLastError();
                return fail(OVL_ECUDA, std::string("wilson_apply_noalloc: cudaGetSymbolAddress failed: ") +
                                           cudaGetErrorString(e));
            }
            g_noalloc_addr[dev] = addr;
        }
        scratch = (unsigned char *)g_noalloc_addr[dev];
    }
    Geom g{};
    for (int m = 0; m < 4; m++) g.L[m] = dims[m];
    g.V = (int)V;
    g.Vh = (int)(V / 2);
    g.Lh3 = dims[3] / 2;
    g.antiperiodic = antiperiodic ? 1 : 0;
    g.tps64 = g.tps32 = 1;
    g.mrhs32 = g.mrhs32l = 1;
    if (cudaDeviceGetAttribute(&g.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(OVL_ECUDA, "wilson_apply_noalloc: cannot query the device");
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double2 *links = (double2 *)scratch;
    double2 *pin = (double2 *)(scratch + kNoAllocLinkBytes);
    double2 *pout = (double2 *)(scratch + kNoAllocLinkBytes + kNoAllocSpinorBytes);
    k_noalloc_pack_links<<<plain_grid(V * 4), kBlock, 0, st>>>(g, (const double2 *)gauge);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = pack_spinor_f64(g, pin, in, st)) != cudaSuccess ||
        (e = wilson_f64(g, links, pin, pout, m0, 0, 1.0, nullptr, 0.0, st)) != cudaSuccess ||
        (e = unpack_spinor_f64(g, out, pout, st)) != cudaSuccess) {
        cudaGetLastError();
        return fail(OVL_ECUDA, std::string("wilson_apply_noalloc: ") + cudaGetErrorString(e));
    }
    return OVL_OK;
}
