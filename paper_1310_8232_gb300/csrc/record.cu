// Recording inside the time loop: receiver traces ("sismic") and the
// discrete wavefield energy after every step (the two steps of Algorithm 1's
// loop body beside the 3D model), both written by the sweep itself.
//
// Traces: the values u^{n+1} of a receiver plane z = rec_z (or one row y of
// it) after each step, as stored (16-bit storage: times the plane's scale),
// [record][ny or 1][nx], copied by a small kernel after the step.
// Energy: E^{n+1/2} = sum_p (u^{n+1} - u^n)^2 / kappa - u^{n+1} Lambda(u^n)
// (the quantity the scheme conserves without a source; dx^2 / dt^2 times the
// physical discrete energy), summed inside the sweep: per warp in FP32 over
// a ring of planes, per block in FP64, and over blocks in block order by the
// last block of the launch.
#include <algorithm>

#include "plan_impl.h"

using namespace stencil;

extern "C" {

void stencil_record_cfg_init(stencil_record_cfg *c)
{
    if (!c) return;
    c->receiver_z = -1;
    c->receiver_y = -1;
    c->energy = 0;
    c->capacity = 0;
}

int stencil_record_stop(stencil_plan_t h)
{
    if (!h) return fail(STENCIL_EINVAL, "null plan");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    if (!p->rec_mem) return STENCIL_OK;
    int rc = p->check_device_error();        // no sweep may still write the buffers
    p->drop_graphs();                         // captured launches carry the recording pointers
    p->dev_free(p->rec_mem);
    p->rec_mem = nullptr;
    p->rec = nullptr;
    p->rec_energy = p->rec_part = nullptr;
    p->rec_count = nullptr;
    p->rec_cap = 0;
    p->rec_z = p->rec_y = -1;
    p->rec_energy_on = 0;
    return rc;
}

int stencil_record_start(stencil_plan_t h, const stencil_record_cfg *c)
{
    if (!h || !c) return fail(STENCIL_EINVAL, "null argument");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    if (p->tile.kernel == STENCIL_KERNEL_TWO_STEP)
        return fail(STENCIL_EUNSUPPORTED, "the two-step kernel records nothing (each launch spans two steps)");
    if (c->capacity < 1) return fail(STENCIL_EINVAL, "capacity must be >= 1");
    if (c->receiver_z < -1 || c->receiver_z >= p->nz) return fail(STENCIL_EINVAL, "receiver_z outside the grid");
    if (c->receiver_y < -1 || c->receiver_y >= p->ny) return fail(STENCIL_EINVAL, "receiver_y outside the grid");
    if (c->receiver_z < 0 && !c->energy) return fail(STENCIL_EINVAL, "nothing to record");
    if (c->energy && (p->absorb_w > 0 || p->inj))
        return fail(STENCIL_EUNSUPPORTED, "the energy is recorded for plans without an absorbing layer or injection");
    int rc = stencil_record_stop(h);
    if (rc) return rc;
    const int64_t per = c->receiver_z < 0 ? 0 : (int64_t)(c->receiver_y < 0 ? p->ny : 1) * p->nx;
    // the sweep's grid: one energy partial per block
    int64_t blocks;
    if (p->tile.kernel == STENCIL_KERNEL_NAIVE) {
        // at least its blocks: 128 x 1 each, or narrower and taller on narrow grids
        blocks = (int64_t)((p->nx + 127) / 128) * p->ny * p->nz;
    } else {
        const int zc = p->tile.zchunk > 0 ? p->tile.zchunk : p->nz;
        blocks = (int64_t)((p->nx + p->tile.tx - 1) / p->tile.tx) * ((p->ny + p->tile.ty - 1) / p->tile.ty) *
                 ((p->nz + zc - 1) / zc);
    }
    const size_t e_bytes = c->energy ? sizeof(double) * ((size_t)c->capacity + blocks) + 256 : 0;
    const size_t t_bytes = sizeof(float) * (size_t)per * c->capacity;
    void *mem = nullptr;
    cudaError_t e = p->dev_alloc(&mem, e_bytes + t_bytes);
    if (e != cudaSuccess) return fail(STENCIL_ENOMEM, "recording buffers of %zu bytes", e_bytes + t_bytes);
    char *b = static_cast<char *>(mem);
    p->rec_mem = mem;
    if (c->energy) {
        p->rec_count = reinterpret_cast<unsigned *>(b);
        p->rec_energy = reinterpret_cast<double *>(b + 256);
        p->rec_part = p->rec_energy + c->capacity;
        e = cudaMemsetAsync(b, 0, e_bytes, p->stream);
        // unrecorded steps read back as NaN
        if (e == cudaSuccess) e = cudaMemsetAsync(p->rec_energy, 0xff, sizeof(double) * c->capacity, p->stream);
    }
    p->rec = t_bytes ? reinterpret_cast<float *>(b + e_bytes) : nullptr;
    if (e == cudaSuccess && t_bytes) e = cudaMemsetAsync(p->rec, 0, t_bytes, p->stream);
    if (e != cudaSuccess) {
        stencil_record_stop(h);
        return fail_cuda(e, "recording buffers");
    }
    p->rec_n0 = p->steps_done;
    p->rec_cap = c->capacity;
    p->rec_z = c->receiver_z;
    p->rec_y = c->receiver_y;
    p->rec_energy_on = c->energy ? 1 : 0;
    p->drop_graphs();
    return p->check_device_error();
}

int stencil_record_read(stencil_plan_t h, float *traces, int32_t traces_on_device, double *energy,
                        int32_t *nrecorded)
{
    if (!h) return fail(STENCIL_EINVAL, "null plan");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    if (!p->rec_mem) return fail(STENCIL_EINVAL, "no recording started");
    int rc = p->check_device_error();
    if (rc) return rc;
    const int64_t n = std::max<int64_t>(0, std::min<int64_t>(p->rec_cap, p->steps_done - p->rec_n0));
    if (nrecorded) *nrecorded = (int32_t)n;
    cudaError_t e = cudaSuccess;
    if (traces && p->rec && n) {
        const int64_t per = (int64_t)(p->rec_y < 0 ? p->ny : 1) * p->nx;
        e = cudaMemcpyAsync(traces, p->rec, sizeof(float) * per * n,
                            traces_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream);
    }
    if (e == cudaSuccess && energy && p->rec_energy && n)
        e = cudaMemcpyAsync(energy, p->rec_energy, sizeof(double) * n, cudaMemcpyDeviceToHost, p->stream);
    if (e != cudaSuccess) return fail_cuda(e, "recording read-back");
    e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail_cuda(e, "recording read-back");
    return STENCIL_OK;
}

}  // extern "C"
