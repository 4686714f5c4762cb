// lb.cu -- D3Q19 lattice Boltzmann step (Section 3.3, Eq. 16-21) for sm_103a.
//
// One fused kernel per step: pull streaming from the post-collision buffer
// (periodic x, y; halfway bounce-back at the z walls with the moving-wall
// term at the top), moments (Eq. 17-18), force-corrected velocity
// v = u + F/(2 rho), BGK relaxation to the equilibrium of Eq. 20 and Guo's
// source (Eq. 19 with the (c c^T - c_s^2 I) tensor), written to the other
// buffer.  Populations are stored shifted, f~ = f - w_q, so that FP32 keeps
// the small deviations from rest that carry the flow (|u| ~ 1e-5..1e-3).
//
// Layout: structure of arrays f[q][cell], x fastest; one thread per cell, a
// block covers a run of one (j, k) row so that the wall branch and the row's
// force flag are uniform across the block.  Traffic per cell: 19 float
// loads + 19 float stores (152 B), plus, in rows marked by the spreading
// kernel, the force (16 B read, 16 B cleared) and the velocity (16 B).
#include <climits>

#include "pfsi_internal.cuh"

namespace pfsi {

namespace {

constexpr int kRowBlock = 128;

__global__ void __launch_bounds__(kRowBlock) k_lb_step(
    const float* __restrict__ fin, float* __restrict__ fout, float4* __restrict__ g,
    float4* __restrict__ vout, const uint32_t* __restrict__ flags, int nx, int ny, int nz,
    float omega, float guo, float3 body, float3 utop)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const int N = nx * ny * nz;
    const int row = k * ny + j;
    const int cell = row * nx + i;
    const int xm = (i == 0) ? nx - 1 : i - 1;       // source column for c_x = +1
    const int xp = (i == nx - 1) ? 0 : i + 1;       // source column for c_x = -1
    const int ym = (j == 0) ? ny - 1 : j - 1;
    const int yp = (j == ny - 1) ? 0 : j + 1;

    float f[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const int sx = cxq(q) == 1 ? xm : (cxq(q) == -1 ? xp : i);
        const int sy = cyq(q) == 1 ? ym : (cyq(q) == -1 ? yp : j);
        const int sk = k - czq(q);
        if (czq(q) == 1 && k == 0) {
            f[q] = fin[oppq(q) * N + cell];                         // still bottom wall
        } else if (czq(q) == -1 && k == nz - 1) {
            const float cu = cxq(q) * utop.x + cyq(q) * utop.y;     // moving top wall,
            f[q] = fin[oppq(q) * N + cell] + 6.0f * wq(q) * cu;     // rho_w = 1
        } else {
            f[q] = fin[q * N + (sk * ny + sy) * nx + sx];
        }
    }

    float drho = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        drho += f[q];
        if (cxq(q)) mx += cxq(q) * f[q];
        if (cyq(q)) my += cyq(q) * f[q];
        if (czq(q)) mz += czq(q) * f[q];
    }
    const float rho = 1.0f + drho;
    float Fx = body.x, Fy = body.y, Fz = body.z;
    const bool forced = flags[row] != 0u;
    if (forced) {
        const float4 gg = g[cell];
        Fx += gg.x;
        Fy += gg.y;
        Fz += gg.z;
    }
    const float irho = 1.0f / rho;
    const float vx = (mx + 0.5f * Fx) * irho;
    const float vy = (my + 0.5f * Fy) * irho;
    const float vz = (mz + 0.5f * Fz) * irho;
    const float vv = vx * vx + vy * vy + vz * vz;
    const float vF = vx * Fx + vy * Fy + vz * Fz;

#pragma unroll
    for (int q = 0; q < 19; ++q) {
        float cv = 0.f, cF = 0.f;
        if (cxq(q)) { cv += cxq(q) * vx; cF += cxq(q) * Fx; }
        if (cyq(q)) { cv += cyq(q) * vy; cF += cyq(q) * Fy; }
        if (czq(q)) { cv += czq(q) * vz; cF += czq(q) * Fz; }
        // equilibrium minus w_q (Eq. 20, shifted storage)
        const float feq = wq(q) * (drho + rho * (3.0f * cv + 4.5f * cv * cv - 1.5f * vv));
        // Guo: w (1 - 1/2tau) [3 c.F + 9 (c.v)(c.F) - 3 v.F]
        const float src = wq(q) * guo * (3.0f * cF + 9.0f * cv * cF - 3.0f * vF);
        fout[q * N + cell] = f[q] + omega * (feq - f[q]) + src;
    }
    if (forced) {
        vout[cell] = make_float4(vx, vy, vz, rho);
        g[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Developed shear profile, post-collision, shifted by w_q; evaluated in FP64.
__global__ void k_lb_init_shear(float* __restrict__ f, int nx, int ny, int nz, double tau,
                                double ux_top, double uy_top)
{
    const int N = nx * ny * nz;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < N; cell += gridDim.x * blockDim.x) {
        const int k = cell / (nx * ny);
        const double dux = ux_top / nz, duy = uy_top / nz;
        const double ux = dux * (k + 0.5), uy = duy * (k + 0.5);
        const double uu = ux * ux + uy * uy;
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            const double w = q < 6 ? 1.0 / 18.0 : (q < 18 ? 1.0 / 36.0 : 1.0 / 3.0);
            const double cu = cxq(q) * ux + cyq(q) * uy;
            const double feq = w * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            const double qgrad = (double)czq(q) * (cxq(q) * dux + cyq(q) * duy);
            const double fneq_post = -(tau - 1.0) * w * 3.0 * qgrad;
            f[q * N + cell] = (float)(feq + fneq_post);
        }
    }
}

// FP64 sums of rho and rho*u of the current state.
__global__ void k_lb_moments(const float* __restrict__ f, int N, double* __restrict__ acc)
{
    double s[4] = {0, 0, 0, 0};
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < N; cell += gridDim.x * blockDim.x) {
        double d = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            const double fq = (double)f[q * N + cell];
            d += fq;
            mx += cxq(q) * fq;
            my += cyq(q) * fq;
            mz += czq(q) * fq;
        }
        s[0] += 1.0 + d;
        s[1] += mx;
        s[2] += my;
        s[3] += mz;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double x = s[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&acc[c], x);
    }
}

}  // namespace

int launch_lb_step(LbCtx* c, cudaStream_t s)
{
    const lb_params& p = c->p;
    const int bx = p.nx >= kRowBlock ? kRowBlock : ((p.nx + 31) / 32) * 32;
    const dim3 grid((p.nx + bx - 1) / bx, p.ny, p.nz);
    const float omega = 1.0f / p.tau;
    const float guo = 1.0f - 0.5f / p.tau;
    k_lb_step<<<grid, bx, 0, s>>>(c->f[c->cur], c->f[c->cur ^ 1], c->g, c->v, c->flags, p.nx,
                                  p.ny, p.nz, omega, guo, make_float3(p.body[0], p.body[1], p.body[2]),
                                  make_float3(p.u_top[0], p.u_top[1], p.u_top[2]));
    c->cur ^= 1;
    return check_launch("lb_step");
}

}  // namespace pfsi

using namespace pfsi;

extern "C" int lb_query_sizes(const lb_params* p, lb_sizes* out)
{
    if (!p || !out) return set_error(PFSI_ERR_ARG, "lb_query_sizes: null argument");
    if (p->nx < 1 || p->ny < 1 || p->nz < 2)
        return set_error(PFSI_ERR_ARG, "lb_query_sizes: need nx, ny >= 1 and nz >= 2");
    const long long N = (long long)p->nx * p->ny * p->nz;
    if (N * 19 > (long long)INT_MAX)
        return set_error(PFSI_ERR_ARG, "lb_query_sizes: grid too large (19 * cells must fit in int32)");
    out->n_cells = N;
    out->f_bytes = (size_t)N * 19 * sizeof(float);
    out->g_bytes = (size_t)N * sizeof(float4);
    out->v_bytes = (size_t)N * sizeof(float4);
    out->flag_bytes = (size_t)p->ny * p->nz * sizeof(uint32_t);
    return PFSI_OK;
}

extern "C" int lb_create(const lb_params* p, float* f_a, float* f_b, float* g, float* v,
                         uint32_t* row_flags, lb_ctx** out)
{
    lb_sizes sz;
    int rc = lb_query_sizes(p, &sz);
    if (rc) return rc;
    if (!out || !f_a || !f_b || !g || !v || !row_flags)
        return set_error(PFSI_ERR_ARG, "lb_create: null buffer");
    if (!aligned(f_a, 16) || !aligned(f_b, 16) || !aligned(g, 16) || !aligned(v, 16) || !aligned(row_flags, 4))
        return set_error(PFSI_ERR_ARG, "lb_create: buffers must be 16-byte aligned");
    if (!(p->tau > 0.5f)) return set_error(PFSI_ERR_ARG, "lb_create: tau must exceed 1/2");
    if (p->u_top[2] != 0.0f) return set_error(PFSI_ERR_ARG, "lb_create: the top wall cannot move along z");
    rc = ib_prepare();
    if (rc) return rc;
    lb_ctx* c = new lb_ctx();
    c->p = *p;
    c->N = sz.n_cells;
    c->f[0] = f_a;
    c->f[1] = f_b;
    c->cur = 0;
    c->g = reinterpret_cast<float4*>(g);
    c->v = reinterpret_cast<float4*>(v);
    c->flags = row_flags;
    rc = check_cuda(cudaMemsetAsync(c->g, 0, sz.g_bytes, 0), "lb_create: clear g");
    if (!rc) rc = check_cuda(cudaMemsetAsync(c->flags, 0, sz.flag_bytes, 0), "lb_create: clear flags");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(0), "lb_create: synchronise");
    if (rc) {
        delete c;
        return rc;
    }
    *out = c;
    return PFSI_OK;
}

extern "C" int lb_destroy(lb_ctx* ctx)
{
    delete ctx;
    return PFSI_OK;
}

extern "C" int lb_init_shear(lb_ctx* c, void* stream)
{
    if (!c) return set_error(PFSI_ERR_ARG, "lb_init_shear: null context");
    const int N = (int)c->N;
    const int blocks = (N + 255) / 256 < 148 * 16 ? (N + 255) / 256 : 148 * 16;
    k_lb_init_shear<<<blocks, 256, 0, as_stream(stream)>>>(c->f[c->cur], c->p.nx, c->p.ny, c->p.nz,
                                                           (double)c->p.tau, (double)c->p.u_top[0],
                                                           (double)c->p.u_top[1]);
    return check_launch("lb_init_shear");
}

extern "C" int lb_step(lb_ctx* c, int nsteps, void* stream)
{
    if (!c) return set_error(PFSI_ERR_ARG, "lb_step: null context");
    if (nsteps < 0) return set_error(PFSI_ERR_ARG, "lb_step: negative step count");
    for (int s = 0; s < nsteps; ++s) {
        const int rc = launch_lb_step(c, as_stream(stream));
        if (rc) return rc;
    }
    return PFSI_OK;
}

extern "C" int lb_current(const lb_ctx* c, float** f)
{
    if (!c || !f) return set_error(PFSI_ERR_ARG, "lb_current: null argument");
    *f = c->f[c->cur];
    return PFSI_OK;
}

extern "C" int lb_moments_fp64(lb_ctx* c, double* dev_scratch4, double* out_host, void* stream)
{
    if (!c || !dev_scratch4 || !out_host) return set_error(PFSI_ERR_ARG, "lb_moments_fp64: null argument");
    if (!aligned(dev_scratch4, 8)) return set_error(PFSI_ERR_ARG, "lb_moments_fp64: scratch must be 8-byte aligned");
    cudaStream_t s = as_stream(stream);
    int rc = check_cuda(cudaMemsetAsync(dev_scratch4, 0, 4 * sizeof(double), s), "lb_moments_fp64: clear");
    if (rc) return rc;
    const int N = (int)c->N;
    const int blocks = (N + 255) / 256 < 148 * 8 ? (N + 255) / 256 : 148 * 8;
    k_lb_moments<<<blocks, 256, 0, s>>>(c->f[c->cur], N, dev_scratch4);
    rc = check_launch("lb_moments_fp64");
    if (rc) return rc;
    rc = check_cuda(cudaMemcpyAsync(out_host, dev_scratch4, 4 * sizeof(double), cudaMemcpyDeviceToHost, s),
                    "lb_moments_fp64: copy");
    if (rc) return rc;
    return check_cuda(cudaStreamSynchronize(s), "lb_moments_fp64: synchronise");
}
