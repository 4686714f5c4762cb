// static_scratch.cu -- membrane_measure_static: per-platelet area and volume
// with library-owned scratch, for callers that cannot allocate device memory.
//
// Who needs it: a host application that owns every device allocation (a
// fixed arena handed out by its own allocator, or a real-time loop in which
// cudaMalloc is forbidden) and still wants the area/volume diagnostics of a
// membrane context it has already built.  membrane_measure accumulates in the
// context's workspace, which the caller sized and allocated; this variant
// accumulates in a file-scope static device array instead and touches nothing
// else of the workspace's scratch (it reads the positions and the context's
// triangles, triangle platelets and anchors only).
//
// The array (kMaxPlatelets x {area, volume} doubles, 128 KiB) exists on every
// GPU that loads this library until the process exits.  Its name, in host
// code, is only a host-side stand-in: the device address is looked up once
// per device with cudaGetSymbolAddress (on the first call made while that
// device is current), kept until the process exits and passed to the
// kernels.  A cudaDeviceReset unloads the module; the address kept from
// before it is then stale, so the entry point must not be used after one.
#include <mutex>

#include "pfsi_internal.cuh"

namespace pfsi {

namespace {

constexpr int kMaxPlatelets = PFSI_STATIC_MAX_PLATELETS;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_measure_scratch[2 * kMaxPlatelets];

std::mutex g_addr_mutex;
double* g_addr[kMaxDevices];  // device address of g_measure_scratch per device

__global__ void k_static_zero(double* __restrict__ acc, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) acc[i] = 0.0;
}

// One thread per triangle: area 0.5 |e1 x e2| and signed tetrahedron volume
// (1/6) (a - o).((b - o) x (c - o)) in FP64, summed per platelet (triangles of
// a platelet are contiguous, so a warp is almost always uniform).
__global__ void __launch_bounds__(256) k_static_measure(const double* __restrict__ X, int n, int nt,
                                                        const int* __restrict__ tri,
                                                        const int* __restrict__ tri_plt,
                                                        const int* __restrict__ anchor,
                                                        double* __restrict__ acc)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    int p = -1;
    double S = 0.0, V = 0.0;
    if (t < nt) {
        p = tri_plt[t];
        const int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2], o = anchor[p];
        double pa[3], pb[3], pc[3];
        for (int d = 0; d < 3; ++d) {
            const double od = X[d * n + o];
            pa[d] = X[d * n + a] - od;
            pb[d] = X[d * n + b] - od;
            pc[d] = X[d * n + c] - od;
        }
        const double e1[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
        const double e2[3] = {pc[0] - pa[0], pc[1] - pa[1], pc[2] - pa[2]};
        const double nn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                              e1[0] * e2[1] - e1[1] * e2[0]};
        S = 0.5 * sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        const double bc[3] = {pb[1] * pc[2] - pb[2] * pc[1], pb[2] * pc[0] - pb[0] * pc[2],
                              pb[0] * pc[1] - pb[1] * pc[0]};
        V = (pa[0] * bc[0] + pa[1] * bc[1] + pa[2] * bc[2]) / 6.0;
    }
    const int p0 = __shfl_sync(0xffffffffu, p, 0);
    if (__all_sync(0xffffffffu, p == p0)) {
        if (p0 >= 0) {
            for (int off = 16; off > 0; off >>= 1) {
                S += __shfl_down_sync(0xffffffffu, S, off);
                V += __shfl_down_sync(0xffffffffu, V, off);
            }
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(&acc[2 * p0], S);
                atomicAdd(&acc[2 * p0 + 1], V);
            }
        }
    } else if (p >= 0) {
        atomicAdd(&acc[2 * p], S);
        atomicAdd(&acc[2 * p + 1], V);
    }
}

// Device address of the static scratch on the current device.
int scratch_address(double** out)
{
    int dev = 0;
    int rc = check_cuda(cudaGetDevice(&dev), "membrane_measure_static: current device");
    if (rc) return rc;
    if (dev < 0 || dev >= kMaxDevices) return set_error(PFSI_ERR_ARG, "membrane_measure_static: device index too large");
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        rc = check_cuda(cudaGetSymbolAddress(&p, g_measure_scratch), "membrane_measure_static: scratch address");
        if (rc) return rc;
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return PFSI_OK;
}

}  // namespace

}  // namespace pfsi

using namespace pfsi;

extern "C" int membrane_measure_static(mem_ctx* c, const double* X, double* out_host, void* stream)
{
    if (!c || !X || !out_host) return set_error(PFSI_ERR_ARG, "membrane_measure_static: null argument");
    if (!aligned(X, 8)) return set_error(PFSI_ERR_ARG, "membrane_measure_static: misaligned positions");
    if (c->nplt > kMaxPlatelets)
        return set_error(PFSI_ERR_ARG, "membrane_measure_static: " + std::to_string(c->nplt) +
                                           " platelets exceed the static scratch (at most " +
                                           std::to_string(kMaxPlatelets) + ")");
    double* acc = nullptr;
    int rc = scratch_address(&acc);
    if (rc) return rc;
    cudaStream_t s = as_stream(stream);
    const int nacc = 2 * c->nplt;
    k_static_zero<<<(nacc + 255) / 256, 256, 0, s>>>(acc, nacc);
    rc = check_launch("membrane_measure_static: clear scratch");
    if (rc) return rc;
    if (c->nt > 0) {
        k_static_measure<<<(c->nt + 255) / 256, 256, 0, s>>>(X, c->n, c->nt, c->tri, c->tri_plt, c->plt_anchor, acc);
        rc = check_launch("membrane_measure_static: reduction");
        if (rc) return rc;
    }
    rc = check_cuda(cudaMemcpyAsync(out_host, acc, sizeof(double) * nacc, cudaMemcpyDeviceToHost, s),
                    "membrane_measure_static: copy");
    if (rc) return rc;
    return check_cuda(cudaStreamSynchronize(s), "membrane_measure_static: synchronise");
}
