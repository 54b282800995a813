// noalloc.cu -- an entry point that performs M = m^2 - D_eo D_oe without
// allocating any device memory.
//
// stag_apply_M needs an odd-parity intermediate t = D_oe in; a context
// allocates it with cudaMalloc when it is created.  Some callers cannot do
// that: hosts that own every device byte through their own pre-sized arena
// or caching allocator and forbid a library to allocate behind it, and
// latency-critical loops that cannot absorb the device-wide synchronisation
// cudaFree implies (or the latency of cudaMalloc).  For them this variant takes
// the gauge field straight from the caller's canonical buffer (no context, no
// internal link copy) and keeps the intermediate in a fixed, statically sized
// device array that is part of the loaded library image.
//
// The array holds STAG_NOALLOC_MAX_VH x 3 complex doubles (6 MiB) on every GPU
// that loads the library, until the process exits.  Every call shares it:
// calls that overlap on the GPU (different streams, or different host threads
// on one device) race on it and must be serialised by the caller.  The array
// keeps the previous call's contents; each call overwrites every element it
// reads before reading it, so nothing has to start at zero.
#include <mutex>

#include "cg_kernels.cuh"

namespace stag {

static __device__ __align__(256) double2 g_noalloc_odd[(size_t)STAG_NOALLOC_MAX_VH * 3];

// Links read directly from the canonical layout U[i][mu][a][b] (complex128):
// the lexicographic index i of half site h of parity par is rebuilt from its
// coordinates.
struct LinkCanonicalF64 {
    typedef double real;
    typedef double2 store;
    const double2* U;
    Geom g;
    __device__ __forceinline__ Mat3<double> load(int par, int mu, int h) const
    {
        const int r = h / g.Lxh;
        const int xh = h - r * g.Lxh;
        const int y = r % g.L[1];
        const int zt = r / g.L[1];
        const int z = zt % g.L[2];
        const int t = zt / g.L[2];
        const int x = 2 * xh + ((par + y + z + t) & 1);
        const size_t i = (size_t)x + (size_t)g.L[0] * r;
        const double2* p = U + (i * 4 + mu) * 9;
        Mat3<double> m;
#pragma unroll
        for (int k = 0; k < 9; ++k) m.m[k] = to_cplx(__ldg(p + k));
        return m;
    }
};

// Device address of g_noalloc_odd, looked up once per device with that
// device current (the host-side symbol is only a stand-in, not a device
// address).  The address is cached for the life of the device's primary
// context: a cudaDeviceReset between calls (which unloads the module and may
// reload it elsewhere) is not supported.
static int noalloc_scratch(double2** out)
{
    static std::mutex mu;
    static double2* addr[64] = {};
    int dev = 0;
    STAG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d out of range", dev);
        return STAG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_odd);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
            return STAG_ECUDA;
        }
        addr[dev] = (double2*)p;
    }
    *out = addr[dev];
    return STAG_OK;
}

// A buffer the kernels may dereference: device (or managed) memory of the
// current device.  Memory of another GPU is rejected: the kernels would reach
// it through the unified address space without peer access and fault.
static int check_device_buffer(const void* p, const char* what, int dev)
{
    if (!p || ((uintptr_t)p & 15u)) {
        set_error("%s is NULL or not 16-byte aligned", what);
        return STAG_EINVAL;
    }
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        set_error("%s is not a CUDA pointer", what);
        return STAG_EINVAL;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
        set_error("%s is not device memory", what);
        return STAG_EINVAL;
    }
    if (a.type == cudaMemoryTypeDevice && a.device != dev) {
        set_error("%s lives on device %d, but device %d is current", what, a.device, dev);
        return STAG_EINVAL;
    }
    return STAG_OK;
}

}  // namespace stag

using namespace stag;

extern "C" int stag_apply_M_noalloc(const int dims[4], const double* U, double* out_even, const double* in_even,
                                    double mass, void* stream)
{
    if (!dims) {
        set_error("dims is NULL");
        return STAG_EINVAL;
    }
    for (int mu = 0; mu < 4; ++mu)
        if (dims[mu] < 2 || dims[mu] % 2) {
            set_error("extent %d of direction %d is not even and >= 2", dims[mu], mu);
            return STAG_EGEOM;
        }
    // The product stops growing once it passes the limit, so every partial
    // product stays below 2^18 * 2^31 and cannot overflow.
    long long V = 1;
    for (int mu = 0; mu < 4 && V <= 2LL * STAG_NOALLOC_MAX_VH; ++mu) V *= dims[mu];
    if (V / 2 > STAG_NOALLOC_MAX_VH) {
        set_error("stag_apply_M_noalloc: the lattice exceeds the static scratch limit of %d sites "
                  "(V <= %d); use a context and stag_apply_M instead",
                  STAG_NOALLOC_MAX_VH, 2 * STAG_NOALLOC_MAX_VH);
        return STAG_EINVAL;
    }
    int dev = 0;
    STAG_CUDA_TRY(cudaGetDevice(&dev));
    STAG_TRY(check_device_buffer(U, "U", dev));
    STAG_TRY(check_device_buffer(out_even, "out_even", dev));
    STAG_TRY(check_device_buffer(in_even, "in_even", dev));
    if (out_even == in_even) {
        set_error("out and in must not alias");
        return STAG_EINVAL;
    }
    double2* t = nullptr;
    STAG_TRY(noalloc_scratch(&t));
    const Geom g = make_geom(dims);
    const LinkCanonicalF64 L{(const double2*)U, g};
    constexpr int BS = 128;
    const int grid = (g.Vh + BS - 1) / BS;
    cudaStream_t s = (cudaStream_t)stream;
    k_hop<LinkCanonicalF64, SpinorF64, BS><<<grid, BS, 0, s>>>(g, 1, L, SpinorF64{(double2*)in_even}, SpinorF64{t},
                                                                nullptr, 0);
    k_xpay_hop<LinkCanonicalF64, SpinorF64, SpinorF64, BS><<<grid, BS, 0, s>>>(g, L, SpinorF64{t}, SpinorF64{(double2*)in_even},
                                                                     SpinorF64{(double2*)out_even}, mass * mass);
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}
