// Run resume: an ensemble's run state written to a caller-owned host buffer
// (lbm_ensemble_save) and read back into an ensemble of the same configuration
// (lbm_ensemble_load), so that a long direct-sampling run or a GKTL loop driven
// step by step can stop and continue later with exactly the populations,
// times, drag history, App. D snapshot bank and AMS checkpoints it had.  The
// state is copied in its storage format (FP32 or shifted 16-bit), so a loaded
// ensemble continues bit for bit as the saved one would have.
//
// The byte string is a fixed header followed by sections in a fixed order:
//   int32 t[N], int32 parity[N]        per-clone time and buffer parity
//   populations [N][clone_bytes]       each clone's current buffer, raw
//   double drag[N][tmax]               D history entries 0 .. tmax-1
//   double obs[N][tmax][4]             only with observables enabled
//   snapshots [n_snaps][clone_bytes], double snap_mass[n_snaps]
//   checkpoints [N][n_ck][clone_bytes] n_ck = min(n_ckpt, tmax / stride + 1)
// The header also carries the perturbation mode (lbm_ensemble_set_perturbation).
// Host byte order; the header carries a magic, a version and the total size.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace lbm {
namespace {

constexpr char kMagic[8] = {'L', 'B', 'M', 'R', 'U', 'N', 0, 1};
constexpr uint32_t kVersion = 1;
constexpr int kCfgInts = 18, kCfgDoubles = 9;

struct SaveHeader {
    char magic[8];
    uint32_t version, header_bytes;
    uint64_t total_bytes, seed, clone_bytes;
    double cfg_d[kCfgDoubles];  // the configuration, field by field (lbm_config has padding)
    int32_t n, elem_bytes, pitch, tmax;
    int32_t observe, n_snaps, n_ck, perturb_mode;
    int32_t cfg_i[kCfgInts];
};
static_assert(sizeof(SaveHeader) == 216, "saved-state header layout");

void pack_config(const lbm_config& c, int32_t (&ci)[kCfgInts], double (&cd)[kCfgDoubles])
{
    const int32_t i[kCfgInts] = {c.nx,          c.ny,        c.obs_x0,  c.obs_y0,   c.obs_w,    c.obs_h,
                                 c.storage,     c.shift_exp, c.max_steps, c.ckpt_stride, c.n_snapshots, c.collision,
                                 c.open_x,      c.grid_x0,   c.grid_w,  c.grid_bar, c.grid_gap, c.sponge_len};
    const double d[kCfgDoubles] = {c.tau, c.gx, c.gy, c.init_amp, c.omega_bulk, c.omega_3, c.omega_4, c.u_in,
                                   c.sponge_tau};
    std::memcpy(ci, i, sizeof i);
    std::memcpy(cd, d, sizeof d);
}

struct Layout {
    int32_t tmax, n_ck;
    uint64_t clone_bytes, total;
};

Layout layout(uint64_t clone_bytes, int32_t n, int32_t tmax, bool observe, int32_t n_snaps, int32_t n_ck)
{
    Layout l{tmax, n_ck, clone_bytes, sizeof(SaveHeader)};
    l.total += 2 * sizeof(int32_t) * (uint64_t)n;
    l.total += clone_bytes * (uint64_t)n;
    l.total += sizeof(double) * (uint64_t)n * tmax;
    if (observe) l.total += 4 * sizeof(double) * (uint64_t)n * tmax;
    l.total += (clone_bytes + sizeof(double)) * (uint64_t)n_snaps;
    l.total += clone_bytes * (uint64_t)n * n_ck;
    return l;
}

int32_t checkpoints_saved(const lbm_ensemble* e, int32_t tmax)
{
    return e->n_ckpt > 0 ? std::min(e->n_ckpt, tmax / e->cfg.ckpt_stride + 1) : 0;
}

Layout layout_of(const lbm_ensemble* e)
{
    const int32_t tmax = *std::max_element(e->t_host.begin(), e->t_host.end());
    return layout((uint64_t)e->clone_stride * e->elem_bytes, e->n, tmax, e->observe, e->n_snaps_set,
                  checkpoints_saved(e, tmax));
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" {

int lbm_ensemble_save(lbm_ensemble* e, void* dst, uint64_t capacity, uint64_t* bytes)
{
    if (!e || !bytes) return fail(LBM_ERR_ARG, "lbm_ensemble_save: null argument");
    const Layout l = layout_of(e);
    *bytes = l.total;
    if (!dst) return LBM_OK;
    if (capacity < l.total) return fail(LBM_ERR_ARG, "lbm_ensemble_save: the buffer is smaller than the state");
    SaveHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kMagic, sizeof kMagic);
    h.version = kVersion;
    h.header_bytes = sizeof(SaveHeader);
    h.total_bytes = l.total;
    h.seed = e->seed;
    h.clone_bytes = l.clone_bytes;
    pack_config(e->cfg, h.cfg_i, h.cfg_d);
    h.n = e->n;
    h.elem_bytes = e->elem_bytes;
    h.pitch = e->pitch;
    h.tmax = l.tmax;
    h.observe = e->observe ? 1 : 0;
    h.n_snaps = e->n_snaps_set;
    h.n_ck = l.n_ck;
    h.perturb_mode = e->perturb_mode;
    char* p = static_cast<char*>(dst);
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    std::memcpy(p, e->t_host.data(), sizeof(int32_t) * e->n);
    p += sizeof(int32_t) * e->n;
    std::memcpy(p, e->parity_host.data(), sizeof(int32_t) * e->n);
    p += sizeof(int32_t) * e->n;
    const size_t cb = l.clone_bytes;
    for (int c = 0; c < e->n; ++c, p += cb)
        LBM_CUDA(cudaMemcpyAsync(p, static_cast<const char*>(e->buf[e->parity_host[c]]) + (size_t)c * cb, cb,
                                 cudaMemcpyDeviceToHost, e->stream));
    const size_t row = sizeof(double) * (size_t)l.tmax;
    if (row > 0)
        LBM_CUDA(cudaMemcpy2DAsync(p, row, e->drag, sizeof(double) * e->cfg.max_steps, row, e->n,
                                   cudaMemcpyDeviceToHost, e->stream));
    p += row * e->n;
    if (e->observe) {
        if (row > 0)
            LBM_CUDA(cudaMemcpy2DAsync(p, 4 * row, e->obs, 4 * sizeof(double) * e->cfg.max_steps, 4 * row, e->n,
                                       cudaMemcpyDeviceToHost, e->stream));
        p += 4 * row * e->n;
    }
    if (h.n_snaps > 0) {
        LBM_CUDA(cudaMemcpyAsync(p, e->snaps, cb * h.n_snaps, cudaMemcpyDeviceToHost, e->stream));
        p += cb * h.n_snaps;
        LBM_CUDA(cudaMemcpyAsync(p, e->snap_mass, sizeof(double) * h.n_snaps, cudaMemcpyDeviceToHost, e->stream));
        p += sizeof(double) * h.n_snaps;
    }
    for (int c = 0; c < e->n && l.n_ck > 0; ++c, p += cb * l.n_ck)
        LBM_CUDA(cudaMemcpyAsync(p, static_cast<const char*>(e->ckpt) + (size_t)c * e->n_ckpt * cb, cb * l.n_ck,
                                 cudaMemcpyDeviceToHost, e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    return LBM_OK;
}

int lbm_ensemble_load(lbm_ensemble* e, const void* src, uint64_t bytes)
{
    if (!e || !src) return fail(LBM_ERR_ARG, "lbm_ensemble_load: null argument");
    SaveHeader h;
    if (bytes < sizeof h) return fail(LBM_ERR_ARG, "lbm_ensemble_load: too short for a saved ensemble");
    std::memcpy(&h, src, sizeof h);
    if (std::memcmp(h.magic, kMagic, sizeof kMagic) != 0 || h.header_bytes != sizeof h)
        return fail(LBM_ERR_ARG, "lbm_ensemble_load: not a saved ensemble");
    if (h.version != kVersion) return fail(LBM_ERR_ARG, "lbm_ensemble_load: unknown format version");
    if (h.total_bytes != bytes) return fail(LBM_ERR_ARG, "lbm_ensemble_load: size differs from the saved size");
    int32_t ci[kCfgInts];
    double cd[kCfgDoubles];
    pack_config(e->cfg, ci, cd);
    if (std::memcmp(ci, h.cfg_i, sizeof ci) != 0 || std::memcmp(cd, h.cfg_d, sizeof cd) != 0)
        return fail(LBM_ERR_ARG, "lbm_ensemble_load: the ensemble's configuration differs from the saved one");
    const uint64_t cb = (uint64_t)e->clone_stride * e->elem_bytes;
    if (h.n != e->n || h.elem_bytes != e->elem_bytes || h.pitch != e->pitch || h.clone_bytes != cb)
        return fail(LBM_ERR_ARG, "lbm_ensemble_load: the saved ensemble has another clone count or layout");
    if ((h.observe != 0) != e->observe)
        return fail(LBM_ERR_ARG, "lbm_ensemble_load: enable or disable observables as in the saved ensemble");
    if (e->cnn) return fail(LBM_ERR_STATE, "lbm_ensemble_load: attach the learned score after loading");
    if (h.tmax < 0 || h.tmax > e->cfg.max_steps || h.n_snaps < 0 || h.n_snaps > e->cfg.n_snapshots ||
        h.n_ck != checkpoints_saved(e, h.tmax) || (h.perturb_mode != 0 && h.perturb_mode != 1))
        return fail(LBM_ERR_ARG, "lbm_ensemble_load: inconsistent saved header");
    const Layout l = layout(cb, h.n, h.tmax, h.observe != 0, h.n_snaps, h.n_ck);
    if (l.total != bytes) return fail(LBM_ERR_ARG, "lbm_ensemble_load: inconsistent saved header");
    const char* p = static_cast<const char*>(src) + sizeof h;
    std::vector<int32_t> t(e->n), par(e->n);
    std::memcpy(t.data(), p, sizeof(int32_t) * e->n);
    p += sizeof(int32_t) * e->n;
    std::memcpy(par.data(), p, sizeof(int32_t) * e->n);
    p += sizeof(int32_t) * e->n;
    int32_t tseen = 0;
    for (int c = 0; c < e->n; ++c) {
        if (t[c] < 0 || t[c] > h.tmax || (par[c] != 0 && par[c] != 1))
            return fail(LBM_ERR_ARG, "lbm_ensemble_load: a saved clone time or parity is out of range");
        tseen = std::max(tseen, t[c]);
    }
    if (tseen != h.tmax) return fail(LBM_ERR_ARG, "lbm_ensemble_load: inconsistent saved header");
    // every check passed: overwrite the ensemble
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    for (int c = 0; c < e->n; ++c, p += cb)
        LBM_CUDA(cudaMemcpyAsync(static_cast<char*>(e->buf[par[c]]) + (size_t)c * cb, p, cb, cudaMemcpyHostToDevice,
                                 e->stream));
    const size_t row = sizeof(double) * (size_t)h.tmax;
    if (row > 0)
        LBM_CUDA(cudaMemcpy2DAsync(e->drag, sizeof(double) * e->cfg.max_steps, p, row, row, e->n,
                                   cudaMemcpyHostToDevice, e->stream));
    p += row * e->n;
    if (h.observe) {
        if (row > 0)
            LBM_CUDA(cudaMemcpy2DAsync(e->obs, 4 * sizeof(double) * e->cfg.max_steps, p, 4 * row, 4 * row, e->n,
                                       cudaMemcpyHostToDevice, e->stream));
        p += 4 * row * e->n;
    }
    if (h.n_snaps > 0) {
        LBM_CUDA(cudaMemcpyAsync(e->snaps, p, cb * h.n_snaps, cudaMemcpyHostToDevice, e->stream));
        p += cb * h.n_snaps;
        LBM_CUDA(cudaMemcpyAsync(e->snap_mass, p, sizeof(double) * h.n_snaps, cudaMemcpyHostToDevice, e->stream));
        p += sizeof(double) * h.n_snaps;
    }
    for (int c = 0; c < e->n && h.n_ck > 0; ++c, p += cb * h.n_ck)
        LBM_CUDA(cudaMemcpyAsync(static_cast<char*>(e->ckpt) + (size_t)c * e->n_ckpt * cb, p, cb * h.n_ck,
                                 cudaMemcpyHostToDevice, e->stream));
    LBM_CUDA(cudaMemcpyAsync(e->t_dev, t.data(), sizeof(int32_t) * e->n, cudaMemcpyHostToDevice, e->stream));
    LBM_CUDA(cudaMemcpyAsync(e->parity_dev, par.data(), sizeof(int32_t) * e->n, cudaMemcpyHostToDevice, e->stream));
    // the sticky non-finite and timeout flags belonged to the replaced state
    LBM_CUDA(cudaMemsetAsync(e->flag_dev, 0, sizeof(int32_t) * 3, e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    e->t_host = t;
    e->parity_host = par;
    e->n_snaps_set = h.n_snaps;
    e->seed = h.seed;
    e->perturb_mode = h.perturb_mode;
    e->score_window = 0;  // trailing means are recomputed by lbm_ensemble_scores
    return LBM_OK;
}

}  // extern "C"
