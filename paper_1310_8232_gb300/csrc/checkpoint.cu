// Checkpoint and restore of a plan's time-stepping state.
//
// The state that determines every later step of the leapfrog recursion
// (Sec. 2, Algorithm 1's time loop) is the pair of levels (u^n, u^{n-1}) and
// n itself (the source term reads w(n dt)).  16-bit storage keeps u^n and
// the difference d^n = u^n - u^{n-1} instead, plus the per-plane scales of
// both and their per-plane maxima, from which the scales of level n+1 are
// derived.  A checkpoint holds exactly that, in the storage's own encoding,
// so a restored plan continues bit for bit.
//
// Layout (little-endian, as the host writes it):
//   CkptHeader (128 bytes)
//   u^n              nx*ny*nz elements of esize bytes, dense (x fastest)
//   u^{n-1} (FP32)   same; d^n for 16-bit storage
//   16-bit storage only: scale of u^n, scale of d^n (nz floats each),
//                        amax of u^n,  amax of d^n  (nz uint32 each)
#include <cstring>

#include "plan_impl.h"

namespace stencil {
namespace {

constexpr char MAGIC[8] = {'S', 'T', 'N', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t VERSION = 2;   // 2: 16-bit storage holds (u^n, d^n)

struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int32_t nx, ny, nz, radius;
    int32_t storage, esize;
    int64_t step;
    double dx, dt;
    int32_t src_on, src_x, src_y, src_z;
    double src_f, src_t0, src_scale;
    uint64_t payload_bytes;
    uint8_t reserved[128 - 112];
};
static_assert(sizeof(CkptHeader) == 128, "checkpoint header is 128 bytes");

uint64_t field_bytes(const Plan *p) { return (uint64_t)p->nx * p->ny * p->nz * p->esize; }

uint64_t table_bytes(const Plan *p)
{
    return p->storage == STENCIL_FP32 ? 0 : (uint64_t)p->nz * (2 * sizeof(float) + 2 * sizeof(unsigned));
}

uint64_t total_bytes(const Plan *p) { return sizeof(CkptHeader) + 2 * field_bytes(p) + table_bytes(p); }

int slot_of(int64_t level) { return (int)(((level % 4) + 4) % 4); }

void fill_header(const Plan *p, CkptHeader *h)
{
    std::memset(h, 0, sizeof *h);
    std::memcpy(h->magic, MAGIC, sizeof MAGIC);
    h->version = VERSION;
    h->header_bytes = sizeof *h;
    h->nx = p->nx;
    h->ny = p->ny;
    h->nz = p->nz;
    h->radius = p->R;
    h->storage = p->storage;
    h->esize = p->esize;
    h->step = p->steps_done;
    h->dx = p->dx;
    h->dt = p->dt;
    h->src_on = p->src.on;
    h->src_x = p->src.x;
    h->src_y = p->src.y;
    h->src_z = p->src.z;
    h->src_f = p->src.f;
    h->src_t0 = p->src.t0;
    h->src_scale = p->src.scale;
    h->payload_bytes = total_bytes(p) - sizeof *h;
}

// The pieces of the state after the header: device address, row layout.
struct Piece {
    char *dev;
    size_t dev_pitch, row_bytes, rows;
};

int pieces(Plan *p, Piece out[6], int *n)
{
    const int64_t at = (int64_t)slot_of(p->steps_done) * p->nz;
    int k = 0;
    // u^n, then u^{n-1} (FP32) or d^n (16-bit)
    for (int w = 0; w < 2; ++w)
        out[k++] = {static_cast<char *>(w == 0 || p->storage == STENCIL_FP32 ? p->level_buf(w) : p->dbuf),
                    (size_t)p->pitch * p->esize, (size_t)p->nx * p->esize, (size_t)p->ny * p->nz};
    if (p->storage != STENCIL_FP32) {
        const size_t sb = sizeof(float) * p->nz, ab = sizeof(unsigned) * p->nz;
        out[k++] = {reinterpret_cast<char *>(p->d_scale + at), sb, sb, 1};
        out[k++] = {reinterpret_cast<char *>(p->d_scale_d + at), sb, sb, 1};
        out[k++] = {reinterpret_cast<char *>(p->d_amax + at), ab, ab, 1};
        out[k++] = {reinterpret_cast<char *>(p->d_amax_d + at), ab, ab, 1};
    }
    *n = k;
    return STENCIL_OK;
}

}  // namespace
}  // namespace stencil

using namespace stencil;

extern "C" {

int stencil_checkpoint_size(stencil_plan_t h, uint64_t *bytes)
{
    if (!h || !bytes) return fail(STENCIL_EINVAL, "null argument");
    *bytes = total_bytes(reinterpret_cast<Plan *>(h));
    return STENCIL_OK;
}

int stencil_checkpoint(stencil_plan_t h, void *dst, uint64_t bytes, int32_t on_device)
{
    if (!h || !dst) return fail(STENCIL_EINVAL, "null argument");
    Plan *p = reinterpret_cast<Plan *>(h);
    if (bytes < total_bytes(p)) return fail(STENCIL_EINVAL, "checkpoint buffer of %llu bytes, need %llu",
                                            (unsigned long long)bytes, (unsigned long long)total_bytes(p));
    cudaSetDevice(p->dev);
    // everything enqueued so far must have landed before the state is read
    int rc = p->check_device_error();
    if (rc) return rc;
    CkptHeader hd;
    fill_header(p, &hd);
    const cudaMemcpyKind out = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSuccess;
    if (on_device) e = cudaMemcpyAsync(dst, &hd, sizeof hd, cudaMemcpyHostToDevice, p->stream);
    else std::memcpy(dst, &hd, sizeof hd);
    char *at = static_cast<char *>(dst) + sizeof hd;
    Piece pc[6];
    int n = 0;
    pieces(p, pc, &n);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = memcpy_rows(at, pc[i].row_bytes, pc[i].dev, pc[i].dev_pitch, pc[i].row_bytes, pc[i].rows, out,
                              p->stream);
        at += pc[i].row_bytes * pc[i].rows;
    }
    if (e != cudaSuccess) return fail_cuda(e, "checkpoint copy");
    // the header lives on this stack frame: wait for every copy
    e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail_cuda(e, "checkpoint sync");
    return p->check_device_error();
}

int stencil_restore(stencil_plan_t h, const void *src, uint64_t bytes, int32_t on_device)
{
    if (!h || !src) return fail(STENCIL_EINVAL, "null argument");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    if (bytes < sizeof(CkptHeader)) return fail(STENCIL_EINVAL, "checkpoint shorter than its header");
    CkptHeader hd;
    cudaError_t e = cudaSuccess;
    if (on_device) e = cudaMemcpy(&hd, src, sizeof hd, cudaMemcpyDeviceToHost);
    else std::memcpy(&hd, src, sizeof hd);
    if (e != cudaSuccess) return fail_cuda(e, "checkpoint header read");
    CkptHeader mine;
    fill_header(p, &mine);
    if (std::memcmp(hd.magic, MAGIC, sizeof MAGIC) != 0 || hd.version != VERSION ||
        hd.header_bytes != sizeof hd)
        return fail(STENCIL_EINVAL, "not a checkpoint of this format");
    if (hd.nx != mine.nx || hd.ny != mine.ny || hd.nz != mine.nz || hd.radius != mine.radius ||
        hd.storage != mine.storage || hd.esize != mine.esize)
        return fail(STENCIL_EINVAL, "checkpoint of a %dx%dx%d R=%d storage %d grid, plan is %dx%dx%d R=%d storage %d",
                    hd.nx, hd.ny, hd.nz, hd.radius, hd.storage, mine.nx, mine.ny, mine.nz, mine.radius,
                    mine.storage);
    if (hd.dx != mine.dx || hd.dt != mine.dt || hd.src_on != mine.src_on || hd.src_x != mine.src_x ||
        hd.src_y != mine.src_y || hd.src_z != mine.src_z || hd.src_f != mine.src_f || hd.src_t0 != mine.src_t0 ||
        hd.src_scale != mine.src_scale)
        return fail(STENCIL_EINVAL, "checkpoint made with another dx, dt or source");
    if (hd.step < 0 || hd.payload_bytes != mine.payload_bytes || bytes < total_bytes(p))
        return fail(STENCIL_EINVAL, "checkpoint payload of %llu bytes, plan needs %llu",
                    (unsigned long long)hd.payload_bytes, (unsigned long long)mine.payload_bytes);
    // the levels restored are the ones set_fields would make current
    p->steps_done = hd.step;
    Piece pc[6];
    int n = 0;
    pieces(p, pc, &n);
    const char *at = static_cast<const char *>(src) + sizeof hd;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = memcpy_rows(pc[i].dev, pc[i].dev_pitch, at, pc[i].row_bytes, pc[i].row_bytes, pc[i].rows, kind,
                              p->stream);
        at += pc[i].row_bytes * pc[i].rows;
    }
    if (e == cudaSuccess && p->d_amax) {
        // the maxima of the next two levels are accumulated from zero
        for (int64_t level = hd.step + 1; level <= hd.step + 2 && e == cudaSuccess; ++level) {
            e = cudaMemsetAsync(p->d_amax + (int64_t)slot_of(level) * p->nz, 0, sizeof(unsigned) * p->nz, p->stream);
            if (e == cudaSuccess)
                e = cudaMemsetAsync(p->d_amax_d + (int64_t)slot_of(level) * p->nz, 0, sizeof(unsigned) * p->nz,
                                    p->stream);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_step, &hd.step, sizeof hd.step, cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return fail_cuda(e, "restore copy");
    // hd is on this stack frame and the caller may free src on return
    e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail_cuda(e, "restore sync");
    return p->check_device_error();
}

}  // extern "C"
