// pwa_nll_grad_noalloc: the direct-form NLL + gradient for callers that
// cannot allocate device memory (see include/pwa.h for the contract).
//
// The kernel is the one the context path launches (k_nll_amp.cu); only its
// scratch differs. Instead of a context-owned cudaMalloc buffer it uses the
// file-scope array below, which every GPU that loads the library holds until
// the process exits. Host code must not pass the array's name to a kernel (in
// host code it is a stand-in, not a device address): on the first call on a
// device, with that device current, cudaGetSymbolAddress gives the device
// address, which is cached per device and passed to the kernel.
#include <mutex>

#include "pwa_internal.cuh"

namespace {

// Largest grid the static scratch serves (one persistent CTA per SM; GPUs
// with more SMs simply run 256 CTAs).
constexpr int kNoAllocMaxGrid = 256;

// Partials of up to kNoAllocMaxGrid CTAs as the kernel lays them out, then
// the control words (about 199 KB; the array is 216 KB).
constexpr size_t kNoAllocScratchBytes = 216 * 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
    int num_sms = 0;
};

DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current.
cudaError_t setup_device(int dev, DeviceSetup **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &d = g_setup[dev];
    if (!d.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return e;
        e = pwa::amp_configure();
        if (e != cudaSuccess)
            return e;
        d.scratch = static_cast<unsigned char *>(p);
        d.num_sms = sms;
        d.ready = true;
    }
    *out = &d;
    return cudaSuccess;
}

}  // namespace

extern "C" int pwa_nll_grad_noalloc(const float *d_planes, int64_t plane_pitch, int64_t n_events,
                                    int n_waves, const float *d_amax, const double *d_M,
                                    const double *d_V, double *d_nll, double *d_grad,
                                    int *d_status, void *stream)
{
    if (!d_planes || !d_amax || !d_M || !d_V || !d_nll)
        return PWA_EINVAL;
    if (n_waves < 1 || n_waves > pwa::kMaxWaves)
        return PWA_EINVAL;
    if (n_events < 1 || n_events > ((int64_t)1 << 31) - 1024)
        return PWA_EINVAL;
    if (plane_pitch < n_events || plane_pitch % 4 != 0 ||
        (reinterpret_cast<uintptr_t>(d_planes) & 15) != 0)
        return PWA_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return PWA_ECUDA;
    }
    DeviceSetup *d = nullptr;
    if (setup_device(dev, &d) != cudaSuccess) {
        cudaGetLastError();
        return PWA_ECUDA;
    }
    const int grid = d->num_sms < kNoAllocMaxGrid ? d->num_sms : kNoAllocMaxGrid;
    if (pwa::amp_scratch_bytes_for_grid(grid) > kNoAllocScratchBytes)
        return PWA_ENOTSUP;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The array keeps the previous call's contents: the kernel's work flags,
    // the ticket and the fallback status word must start at zero (the
    // partials are fully overwritten by every call).
    unsigned char *ctl = d->scratch + pwa::amp_flags_offset(grid);  // [flags 16][ticket 8][status 8]
    if (cudaMemsetAsync(ctl, 0, 64, s) != cudaSuccess) {
        cudaGetLastError();
        return PWA_ECUDA;
    }
    CUtensorMap map;
    pwa::Planes planes{const_cast<float *>(d_planes), plane_pitch, n_events, n_waves};
    if (pwa::encode_planes_map(&map, d_planes, n_events, plane_pitch, 2 * n_waves,
                               pwa::amp_box_events(n_waves), pwa::amp_box_rows(n_waves)) !=
        cudaSuccess)
        return PWA_EINVAL;
    pwa::EvalArgs a{};
    a.n_waves = n_waves;
    a.n_events = n_events;
    a.V = d_V;
    a.M = d_M;
    a.amax = d_amax;
    a.partials = reinterpret_cast<double *>(d->scratch);
    a.ticket = reinterpret_cast<unsigned *>(ctl + 16);
    a.status = d_status ? d_status : reinterpret_cast<int *>(ctl + 24);
    a.done = nullptr;
    a.nll = d_nll;
    a.grad = d_grad;
    if (pwa::launch_nll_amp_grid(planes, &map, a, grid, s) != cudaSuccess) {
        cudaGetLastError();
        return PWA_ECUDA;
    }
    return PWA_OK;
}
