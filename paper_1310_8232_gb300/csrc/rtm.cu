// Plane injection and the imaging condition: the pieces reverse-time
// migration adds around the 3D-model sweep (the backward propagation of the
// recorded traces and the zero-lag cross-correlation with the source
// wavefield).  The injection runs as a small kernel after each step
// (plane_ops.cu); these entry points set it up and run the imaging kernel.
#include "plan_impl.h"

using namespace stencil;

extern "C" {

int stencil_inject_stop(stencil_plan_t h)
{
    if (!h) return fail(STENCIL_EINVAL, "null plan");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    if (!p->inj) return STENCIL_OK;
    int rc = p->check_device_error();          // no sweep may still read the data
    p->drop_graphs();                           // captured launches carry the injection
    p->inj = nullptr;
    p->inj_steps = 0;
    p->inj_z = p->inj_y = -1;
    return rc;
}

int stencil_inject_start(stencil_plan_t h, const stencil_inject_cfg *c)
{
    if (!h || !c || !c->data) return fail(STENCIL_EINVAL, "null argument");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    if (p->storage != STENCIL_FP32) return fail(STENCIL_EUNSUPPORTED, "injection needs FP32 storage");
    if (p->tile.kernel == STENCIL_KERNEL_TWO_STEP)
        return fail(STENCIL_EUNSUPPORTED, "the two-step kernel injects nothing (each launch spans two steps)");
    if (c->z < 0 || c->z >= p->nz) return fail(STENCIL_EINVAL, "injection plane outside the grid");
    if (c->y < -1 || c->y >= p->ny) return fail(STENCIL_EINVAL, "injection row outside the grid");
    if (c->steps < 1) return fail(STENCIL_EINVAL, "steps must be >= 1");
    if (p->rec_mem && p->rec_energy_on)
        return fail(STENCIL_EUNSUPPORTED, "the energy is recorded for plans without injection");
    if (!std::isfinite(c->scale)) return fail(STENCIL_EINVAL, "scale must be finite");
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, c->data) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(STENCIL_EINVAL, "injection data must be device memory");
    }
    int rc = stencil_inject_stop(h);
    if (rc) return rc;
    p->inj = c->data;
    p->inj_n0 = p->steps_done;
    p->inj_steps = c->steps;
    p->inj_reverse = c->reverse ? 1 : 0;
    p->inj_z = c->z;
    p->inj_y = c->y;
    p->inj_scale = c->scale;
    p->drop_graphs();
    return STENCIL_OK;
}

int stencil_image_accumulate(stencil_plan_t h, const float *snapshot, float *image, float scale)
{
    if (!h || !snapshot || !image) return fail(STENCIL_EINVAL, "null argument");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    const float *u = nullptr;
    int rc = p->fp32_level(0, &u);
    if (rc) return rc;
    cudaError_t e = launch_image_accumulate(snapshot, u, image, p->nx, p->ny, p->nz, p->pitch, scale, p->stream);
    if (e != cudaSuccess) return fail_cuda(e, "imaging condition");
    return STENCIL_OK;
}

}  // extern "C"
