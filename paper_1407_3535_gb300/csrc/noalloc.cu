// zncc_full_noalloc: the exhaustive search with no device allocation at all.
//
// Some callers cannot allocate device memory while they search: code running
// under a framework allocator that has already reserved the device heap,
// real-time loops where cudaMalloc/cudaFree (which may synchronise the whole
// device) would stall other streams, or embedded users with a fixed memory
// budget.  This entry point serves them: its scratch lives in one file-scope
// __device__ array, sized for a stated maximum problem and held by every GPU
// that loads the library until the process exits.
//
// Host code never dereferences the array's name (on the host it is only a
// stand-in symbol); the device address is looked up once per device with
// cudaGetSymbolAddress, on that device, the first time the entry point runs
// there.  No call may be made while its stream is being captured into a
// graph: every call reads its result back into host memory and waits for
// the stream.  All calls share the one array: anything that must start at zero is cleared
// by the kernels that use it, and calls that overlap on the GPU (for example
// from two streams) race on the shared scratch and must be serialised by the
// caller.
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace opta {
namespace {

// Stated maximum: p, q <= 4096 with p*q <= 2^18 pixels (e.g. 512 x 512), and
// templates with m * round_up(n, 8) <= 4096 elements (e.g. 64 x 64).
constexpr int kNaMaxSide = 4096;
constexpr int64_t kNaMaxPixels = (int64_t)1 << 18;
constexpr int kNaMaxTmpl = 4096;

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct NaLayout {
    size_t i8, stage, iis, iiq, inv, ef, map, tf, td, tstage, cand, crho, st, bad, total;
};

constexpr NaLayout na_layout() {
    NaLayout l{};
    const size_t P = (size_t)kNaMaxPixels;
    const size_t II = P + 2 * (size_t)kNaMaxSide + 1;   // (p+1)(q+1) <= pq + p + q + 1
    const size_t T = (size_t)kNaMaxTmpl;
    size_t o = 0;
    l.i8 = o;     o += al256(P);
    l.stage = o;  o += al256(4 * P);
    l.iis = o;    o += al256(8 * II);
    l.iiq = o;    o += al256(8 * II);
    l.inv = o;    o += al256(4 * P);
    l.ef = o;     o += al256(4 * P);
    l.map = o;    o += al256(4 * P);
    l.tf = o;     o += al256(4 * T);
    l.td = o;     o += al256(8 * T);
    l.tstage = o; o += al256(4 * T);
    l.cand = o;   o += al256(4 * P);
    l.crho = o;   o += al256(8 * P);
    l.st = o;     o += al256(sizeof(TmplState));
    l.bad = o;    o += al256(sizeof(int));
    l.total = o;
    return l;
}
constexpr NaLayout kLay = na_layout();

// The scratch (about 12 MB) of every no-alloc call on this device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kLay.total];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once).
opta_status scratch_address(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return OPTA_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return OPTA_ERR_CUDA;
        }
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return OPTA_OK;
}

opta_status na_err(cudaError_t e) {
    if (e == cudaSuccess) return OPTA_OK;
    cudaGetLastError();
    return OPTA_ERR_CUDA;
}

}  // namespace
}  // namespace opta

using namespace opta;

extern "C" opta_status zncc_full_noalloc(const opta_image *img, const opta_template *t,
                                         float *rho_map, opta_result *best, void *stream) {
    if (!img || !img->data || !t || !t->data || !best) return OPTA_ERR_INVALID_ARG;
    const int p = img->rows, q = img->cols, m = t->rows, n = t->cols;
    if (p < 1 || q < 1 || img->stride_elems < q || (img->dtype != OPTA_U8 && img->dtype != OPTA_F32) ||
        m < 1 || n < 1 || m > p || n > q || t->stride_elems < n)
        return OPTA_ERR_INVALID_ARG;
    const int npad = (n + 7) & ~7;
    if (p > kNaMaxSide || q > kNaMaxSide || (int64_t)p * q > kNaMaxPixels ||
        (int64_t)m * npad > kNaMaxTmpl)
        return OPTA_ERR_TOO_LARGE;
    unsigned char *base = nullptr;
    const opta_status sa = scratch_address(&base);
    if (sa != OPTA_OK) return sa;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *I8 = base + kLay.i8;
    float *stage = reinterpret_cast<float *>(base + kLay.stage);
    long long *IIS = reinterpret_cast<long long *>(base + kLay.iis);
    long long *IIQ = reinterpret_cast<long long *>(base + kLay.iiq);
    float *inv = reinterpret_cast<float *>(base + kLay.inv);
    float *ef = reinterpret_cast<float *>(base + kLay.ef);
    float *map = rho_map ? rho_map : reinterpret_cast<float *>(base + kLay.map);
    float *tf = reinterpret_cast<float *>(base + kLay.tf);
    double *td = reinterpret_cast<double *>(base + kLay.td);
    float *tst = reinterpret_cast<float *>(base + kLay.tstage);
    int *cand = reinterpret_cast<int *>(base + kLay.cand);
    double *crho = reinterpret_cast<double *>(base + kLay.crho);
    TmplState *st = reinterpret_cast<TmplState *>(base + kLay.st);
    int *bad = reinterpret_cast<int *>(base + kLay.bad);
    cudaError_t e;
#define NA(x) do { if ((e = (x)) != cudaSuccess) return na_err(e); } while (0)
    // image -> uint8 (pixels must be integers in [0, 255])
    if (img->dtype == OPTA_U8) {
        if (img->on_device)
            NA(launch_ingest_u8(static_cast<const uint8_t *>(img->data), img->stride_elems, p, q, I8, s));
        else
            NA(cudaMemcpy2DAsync(I8, q, img->data, img->stride_elems, q, p, cudaMemcpyHostToDevice, s));
    } else {
        const float *src = static_cast<const float *>(img->data);
        int64_t ld = img->stride_elems;
        if (!img->on_device) {
            NA(cudaMemcpy2DAsync(stage, (size_t)q * sizeof(float), src, ld * sizeof(float),
                                 (size_t)q * sizeof(float), p, cudaMemcpyHostToDevice, s));
            src = stage;
            ld = q;
        }
        NA(cudaMemsetAsync(bad, 0, sizeof(int), s));
        NA(launch_ingest_f32(src, ld, p, q, I8, bad, s));
        int hbad = 0;
        NA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        NA(cudaStreamSynchronize(s));
        if (hbad) return OPTA_ERR_UNSUPPORTED;
    }
    const float *tdev = t->data;
    int64_t tld = t->stride_elems;
    if (!t->on_device) {
        NA(cudaMemcpy2DAsync(tst, (size_t)n * sizeof(float), t->data, (size_t)t->stride_elems * sizeof(float),
                             (size_t)n * sizeof(float), m, cudaMemcpyHostToDevice, s));
        tdev = tst;
        tld = n;
    }
#undef NA
    // the same steps as zncc_full, on the static scratch
    const ExhaustiveBufs bufs{IIS, IIQ, inv, ef, map, tf, td, cand, crho, st};
    return exhaustive_run(I8, p, q, tdev, tld, m, n, bufs, best, s);
}
