// gs_api.cu -- the extern "C" entry points of include/gs_topk.h: argument checks,
// workspace layout, camera tables and the launch sequence of each stage.
#include "gs_internal.cuh"

#include <string.h>

#include <algorithm>
#include <mutex>

#ifndef GS_BUILT_SM
#define GS_BUILT_SM 0
#endif

namespace gs {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static bool tile_ok(int tw, int th)
{
    return (tw == 16 && th == 16) || (tw == 32 && th == 8) || (tw == 16 && th == 8) || (tw == 8 && th == 8);
}

bool cfg_ok(const gs_config *cfg)
{
    return cfg && cfg->K >= 1 && cfg->K <= GS_MAX_K && cfg->D >= 8 && cfg->D <= 1024 && cfg->D % 8 == 0 &&
           tile_ok(cfg->tile_w, cfg->tile_h) && (cfg->feat_dtype == GS_F32 || cfg->feat_dtype == GS_BF16) &&
           cfg->max_instances >= 0 && cfg->max_feature_rows >= 0 &&
           (cfg->topk_layout == 0 || (cfg->topk_layout >= 1 && cfg->topk_layout <= 2 && cfg->K <= 16)) &&
           (cfg->depth_cut == 0 || cfg->depth_cut == 1);
}

static bool cams_ok(const gs_camera *cams, int n_cams)
{
    if (!cams || n_cams < 1 || n_cams > GS_MAX_CAMERAS) return false;
    for (int c = 0; c < n_cams; ++c) {
        const gs_camera &k = cams[c];
        if (k.width < 1 || k.height < 1 || k.width > 32768 || k.height > 32768) return false;
        if (!(k.fx > 0.f) || !(k.fy > 0.f) || !(k.near_z > 0.f)) return false;
    }
    return true;
}

bool make_camtable(const gs_config *cfg, const gs_camera *cams, int n_cams, CamTable &ct)
{
    memset(&ct, 0, sizeof(ct));
    ct.n = n_cams;
    ct.tile_w = cfg->tile_w;
    ct.tile_h = cfg->tile_h;
    int tile_off = 0;
    int row_off = 0;
    long long pix_off = 0;
    for (int c = 0; c < n_cams; ++c) {
        const gs_camera &k = cams[c];
        CamDev &d = ct.c[c];
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) d.R[3 * i + j] = k.viewmat[4 * i + j];
            d.t[i] = k.viewmat[4 * i + 3];
        }
        d.fx = k.fx; d.fy = k.fy; d.cx = k.cx; d.cy = k.cy;
        d.near_z = k.near_z;
        d.limx = kFrustumClamp * ((float)k.width / (2.0f * k.fx));
        d.limy = kFrustumClamp * ((float)k.height / (2.0f * k.fy));
        d.W = k.width; d.H = k.height;
        d.tiles_x = (k.width + cfg->tile_w - 1) / cfg->tile_w;
        d.tiles_y = (k.height + cfg->tile_h - 1) / cfg->tile_h;
        d.tile_off = tile_off;
        d.row_off = row_off;
        d.pix_off = pix_off;
        tile_off += d.tiles_x * d.tiles_y;
        row_off += d.tiles_y;
        pix_off += (long long)k.width * k.height;
    }
    ct.n_tiles = tile_off;
    ct.n_rows = row_off;
    return true;
}

bool make_layout(const gs_config *cfg, const gs_camera *cams, int n_cams, int N, WsLayout &L)
{
    if (!cfg_ok(cfg) || !cams_ok(cams, n_cams) || N < 0) return false;
    memset(&L, 0, sizeof(L));
    CamTable ct;
    make_camtable(cfg, cams, n_cams, ct);
    L.N = N; L.K = cfg->K; L.D = cfg->D; L.n_cams = n_cams; L.n_tiles = ct.n_tiles;
    L.depth_cut = cfg->depth_cut != 0;
    // identifies the tile grid the recorded cuts belong to (a first render, or another
    // grid, records and uses none)
    L.cut_sig = 0x9e3779b9u ^ ((uint32_t)ct.n_tiles * 2654435761u) ^ ((uint32_t)cfg->tile_w << 20) ^
                ((uint32_t)cfg->tile_h << 12) ^ (uint32_t)n_cams;
    if (L.cut_sig == 0u) L.cut_sig = 1u;
    L.NE = (long long)n_cams * N;
    L.P = 0;
    for (int c = 0; c < n_cams; ++c) L.P += (long long)cams[c].width * cams[c].height;
    L.PK = L.P * cfg->K;
    long long mcap = cfg->max_instances > 0 ? cfg->max_instances : 32 * L.NE;
    if (mcap < 4096) mcap = 4096;
    if (mcap > 0x7fffffffll) mcap = 0x7fffffffll;
    L.Mcap = mcap;
    L.use_tiles = tile_grad_supported(cfg->feat_dtype, cfg->D, cfg->K);
    CamTable cb;
    const FgBlock fb = fg_block_shape(cfg->feat_dtype, cfg->D, cfg->K);
    if (L.use_tiles) retile(ct, fb.bw, fb.bh, cb);
    L.n_fgblocks = L.use_tiles ? cb.n_tiles : 0;
    // partial feature-gradient rows: one per (block, selected Gaussian), so never more
    // than P K; the configured capacity, else 32 per block, or the instance capacity per
    // element when that is larger (an overflow sets the error word and yields no feature
    // gradient; gs_workspace_counts then reports the rows needed).
    const long long per_block = std::max(32ll, mcap / std::max(1ll, L.NE));
    const long long rows_want = cfg->max_feature_rows > 0 ? (long long)cfg->max_feature_rows
                                                          : (long long)L.n_fgblocks * per_block;
    L.rows_cap = L.use_tiles ? std::min(L.PK, rows_want) : 0;
    L.n_pairs = N + L.rows_cap;
    if (L.NE > 0x7fffffffll || L.n_pairs > 0x7fffffffll) return false;
    L.max_pieces_rows = N + (L.rows_cap + kPieceLen - 1) / kPieceLen + 1;
    L.max_multi_rows = 2 * ((L.rows_cap + kPieceLen - 1) / kPieceLen) + 1;
    L.inst_sorted = sorted_buffer(bits_for(L.n_tiles));
    L.pair_bits = bits_for((long long)N + 1);
    L.pair_sorted = sorted_buffer(L.pair_bits);

    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes > 0 ? bytes : 1); return o; };
    const size_t u = sizeof(uint32_t);
    L.header = take(256);
    for (int i = 0; i < 2; ++i) L.depth_keys[i] = take(u * L.NE);
    for (int i = 0; i < 2; ++i) L.depth_vals[i] = take(u * L.NE);
    L.elem_cnt = take(u * L.NE);
    L.elem_off = take(u * L.NE);
    L.counts = take(u * L.NE);
    L.counts1 = take(u * L.NE);
    for (int i = 0; i < 2; ++i) L.inst_keys[i] = take(u * L.Mcap);
    for (int i = 0; i < 2; ++i) L.inst_vals[i] = take(u * L.Mcap);
    L.inst_elem = take(u * L.Mcap);
    L.tile_range = take(8 * (size_t)L.n_tiles);
    L.tile_range2 = take(8 * (size_t)L.n_tiles);
    L.cut_store = take(u * (size_t)L.n_tiles);
    L.cut_cur = take(u * (size_t)L.n_tiles);
    L.tile_incomplete = take(u * (size_t)L.n_tiles);
    L.tile_sat = take(u * (size_t)L.n_tiles);
    L.cut_rowmin = take(u * (size_t)ct.n_rows);
    L.cut_rowmax = take(u * (size_t)ct.n_rows);
    L.cut_rowmax_st = take(u * (size_t)kCutLevels * ct.n_rows);
    L.sort_hist = take(u * 256 * (kRadixBlocks + 1));
    L.scan_aux = take(u * (kSortBlocks + 32));
    L.inst_grad = take(sizeof(float) * kGradVals * L.Mcap);
    L.inst_walked = take((size_t)L.Mcap);
    L.elem_grad = take(sizeof(float) * kGradVals * L.NE);
    L.pose_part = take(sizeof(float) * 12 * L.NE);
    for (int i = 0; i < 2; ++i) L.pair_keys[i] = take(u * L.n_pairs);
    for (int i = 0; i < 2; ++i) L.pair_vals[i] = take(u * L.n_pairs);
    L.hbuf = take(sizeof(float) * L.PK);
    L.seg_start = take(u * N);
    L.seg_end = take(u * N);
    L.pieces = take(u * N);
    L.piece_off = take(u * N);
    L.multi = take(u * N);
    L.multi_off = take(u * N);
    L.mflag = take(u * N);
    L.mlist = take(u * N);
    L.piece_rank = take(u * L.max_pieces_rows);
    L.piece_rows = take(sizeof(float) * (size_t)L.max_multi_rows * cfg->D);
    L.loss_part = 0;
    if (L.use_tiles) {
        L.tile_keys = take(8 * (size_t)L.n_fgblocks * fb.bw * fb.bh * cfg->K);
        L.tile_runs = take((size_t)L.n_fgblocks * tile_runs_bytes(fb.bw * fb.bh, cfg->K));
        L.tile_u = take(u * L.n_fgblocks);
        L.tile_rowbase = take(u * L.n_fgblocks);
        L.tile_rows = take(sizeof(float) * (size_t)L.rows_cap * cfg->D);
    }
    L.total = off;
    return true;
}

__global__ void k_store_u64(unsigned long long *dst, unsigned long long v) { *dst = v; }

static int ws_check(const WsLayout &L, const void *ws, size_t ws_bytes)
{
    if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < L.total) return GS_ERR_WORKSPACE;
    return GS_OK;
}

static int launch_status()
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

// Kernel timers: one event pair per timed stage, created on first use while enabled.
struct Timers {
    std::mutex m;
    bool enabled = false;
    cudaEvent_t ev[GS_TIMER_COUNT][2] = {};
    bool recorded[GS_TIMER_COUNT] = {};
};
static Timers &timers()
{
    static Timers t;
    return t;
}

TimerScope::TimerScope(int id_, cudaStream_t s_) : id(id_), s(s_), on(false)
{
    Timers &t = timers();
    if (id < 0 || !t.enabled) return;             // (read without the lock: a flag set between renders)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> g(t.m);
    if (!t.ev[id][0] && (cudaEventCreate(&t.ev[id][0]) != cudaSuccess || cudaEventCreate(&t.ev[id][1]) != cudaSuccess)) {
        cudaGetLastError();
        return;
    }
    on = cudaEventRecord(t.ev[id][0], s) == cudaSuccess;
    if (!on) cudaGetLastError();
}

TimerScope::~TimerScope()
{
    if (!on) return;
    Timers &t = timers();
    std::lock_guard<std::mutex> g(t.m);
    if (cudaEventRecord(t.ev[id][1], s) == cudaSuccess) t.recorded[id] = true;
    else cudaGetLastError();
}

// Library-owned auxiliary stream of a device, with the fork and join events of one
// backward call; created on first use, kept until the process exits.
struct AuxStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, hold = nullptr;
};
constexpr int kMaxDevices = 64;

static std::mutex &aux_mutex()
{
    static std::mutex m;
    return m;
}

// The auxiliary stream of the current device, or nullptr (the caller then runs
// everything on its own stream): not yet created while `s` is being captured (a
// creation is not captured work), or creation failed.  Call under aux_mutex().
static const AuxStream *aux_stream(cudaStream_t s)
{
    static AuxStream aux[kMaxDevices];
    static bool failed[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    AuxStream &a = aux[dev];
    if (a.s) return &a;
    if (failed[dev]) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    AuxStream n;
    if (cudaStreamCreateWithFlags(&n.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&n.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&n.join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&n.hold, cudaEventDisableTiming) != cudaSuccess) {
        failed[dev] = true;
        cudaGetLastError();
        return nullptr;
    }
    a = n;
    return &a;
}

}  // namespace gs

using namespace gs;

extern "C" {

const char *gs_status_string(int status)
{
    switch (status) {
    case GS_OK: return "ok";
    case GS_ERR_ARG: return "invalid argument";
    case GS_ERR_WORKSPACE: return "workspace too small or not 256-byte aligned";
    case GS_ERR_CUDA: return "CUDA launch or runtime error";
    case GS_ERR_TIMEOUT: return "a bounded device-side wait ran out";
    case GS_ERR_OVERFLOW: return "instance capacity exceeded (raise gs_config.max_instances)";
    case GS_ERR_UNSUPPORTED: return "configuration not compiled into this library";
    }
    return "unknown status";
}

int gs_version(int *major, int *minor, int *built_sm)
{
    if (major) *major = 0;
    if (minor) *minor = 1;
    if (built_sm) *built_sm = GS_BUILT_SM;
    return GS_OK;
}

size_t gs_workspace_size(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss)
{
    WsLayout L;
    if (!make_layout(cfg, cams, n_cams, n_gauss, L)) return 0;
    return L.total;
}

int64_t gs_pixel_count(const gs_camera *cams, int32_t n_cams)
{
    if (!cams_ok(cams, n_cams)) return -1;
    int64_t P = 0;
    for (int c = 0; c < n_cams; ++c) P += (int64_t)cams[c].width * cams[c].height;
    return P;
}

int gs_preprocess(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                  const float *mean3d, const float *cov3d, const float *opacity, const float *rgb,
                  float *proj, void *ws, size_t ws_bytes, void *stream)
{
    WsLayout L;
    if (!make_layout(cfg, cams, n_cams, n_gauss, L)) return GS_ERR_ARG;
    if (n_gauss > 0 && (!mean3d || !cov3d || !opacity || !rgb || !proj)) return GS_ERR_ARG;
    if (((uintptr_t)proj & 15) != 0) return GS_ERR_ARG;
    int st = ws_check(L, ws, ws_bytes);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CamTable ct;
    make_camtable(cfg, cams, n_cams, ct);
    cudaMemsetAsync(ws_ptr<char>(ws, L.header), 0, 16, s);
    cudaMemsetAsync(ws_ptr<char>(ws, L.header + kHdrWaitLimitByte), 0, 8, s);   // default wait bound
    launch_preprocess(ct, n_gauss, mean3d, cov3d, opacity, rgb, proj, s);
    return launch_status();
}

int gs_bin_sort(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                const float *proj, void *ws, size_t ws_bytes, void *stream)
{
    WsLayout L;
    if (!make_layout(cfg, cams, n_cams, n_gauss, L)) return GS_ERR_ARG;
    if (n_gauss > 0 && !proj) return GS_ERR_ARG;
    int st = ws_check(L, ws, ws_bytes);
    if (st) return st;
    CamTable ct;
    make_camtable(cfg, cams, n_cams, ct);
    launch_bin_sort(ct, L, n_gauss, proj, ws, (cudaStream_t)stream);
    return launch_status();
}

int gs_topk_select(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                   const float *proj, void *ws, size_t ws_bytes,
                   float *rgb_out, float *depth_out, float *T_final, int32_t *n_contrib,
                   int32_t *topk_idx, float *topk_w, void *stream)
{
    WsLayout L;
    if (!make_layout(cfg, cams, n_cams, n_gauss, L)) return GS_ERR_ARG;
    if ((n_gauss > 0 && !proj) || !rgb_out || !depth_out || !T_final || !n_contrib || !topk_idx || !topk_w)
        return GS_ERR_ARG;
    int st = ws_check(L, ws, ws_bytes);
    if (st) return st;
    CamTable ct;
    make_camtable(cfg, cams, n_cams, ct);
    cudaStream_t s = (cudaStream_t)stream;
    if (!launch_walk_fwd(ct, L, cfg->K, cfg->topk_layout, n_gauss, proj, ws, rgb_out, depth_out, T_final, n_contrib,
                         topk_idx, topk_w, 1, s))
        return GS_ERR_UNSUPPORTED;
    if (L.depth_cut) {
        // the tiles the depth cut left unsaturated: their remaining instances, then a
        // second walk over their whole lists (no-ops when none was flagged)
        TimerScope tm(GS_TIMER_COMPLETE, s);
        launch_complete_lists(ct, L, n_gauss, proj, ws, s);
        launch_walk_fwd(ct, L, cfg->K, cfg->topk_layout, n_gauss, proj, ws, rgb_out, depth_out, T_final, n_contrib,
                        topk_idx, topk_w, 2, s);
    }
    return launch_status();
}

int gs_feature_blend(const gs_config *cfg, int64_t n_pix, int32_t n_gauss, const int32_t *topk_idx,
                     const float *topk_w, const void *feats, void *F_out, void *stream)
{
    if (!cfg_ok(cfg) || n_pix < 0 || n_gauss < 0) return GS_ERR_ARG;
    if (n_pix > 0 && (!topk_idx || !topk_w || !F_out)) return GS_ERR_ARG;
    if (n_gauss > 0 && !feats) return GS_ERR_ARG;
    if (((uintptr_t)feats & 15) != 0 || ((uintptr_t)F_out & 15) != 0) return GS_ERR_ARG;
    if (!launch_blend(cfg->feat_dtype, cfg->K, cfg->D, n_pix, n_gauss, topk_idx, topk_w, feats, F_out, nullptr,
                      (cudaStream_t)stream))
        return GS_ERR_UNSUPPORTED;
    return launch_status();
}

int gs_backward(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                const float *mean3d, const float *cov3d, const float *opacity, const float *rgb,
                const void *feats, const float *proj,
                const float *rgb_out, const float *depth_out, const int32_t *topk_idx, const float *topk_w,
                const void *dL_dF, const float *dL_dC, const float *dL_dD,
                const gs_grads *grads, void *ws, size_t ws_bytes, void *stream)
{
    return gs_backward_ex(cfg, cams, n_cams, n_gauss, mean3d, cov3d, opacity, rgb, feats, proj, rgb_out, depth_out,
                          topk_idx, topk_w, dL_dF, dL_dC, dL_dD, grads, 0u, ws, ws_bytes, stream);
}

int gs_backward_ex(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                   const float *mean3d, const float *cov3d, const float *opacity, const float *rgb,
                   const void *feats, const float *proj,
                   const float *rgb_out, const float *depth_out, const int32_t *topk_idx, const float *topk_w,
                   const void *dL_dF, const float *dL_dC, const float *dL_dD,
                   const gs_grads *grads, uint32_t flags, void *ws, size_t ws_bytes, void *stream)
{
    if (flags & ~(uint32_t)GS_BWD_H_FROM_LOSS) return GS_ERR_ARG;
    WsLayout L;
    if (!make_layout(cfg, cams, n_cams, n_gauss, L)) return GS_ERR_ARG;
    // dL_dF == NULL: geometry-only adjoint (no feature loss): no feature gradient, no
    // feature term in dL/dw; feats and grads->feat are then not used
    const bool with_feature = dL_dF != nullptr;
    if (!grads || !rgb_out || !depth_out || !topk_idx || !topk_w || !dL_dC || !dL_dD) return GS_ERR_ARG;
    if (n_gauss > 0 && (!mean3d || !cov3d || !opacity || !rgb || !proj || !grads->opacity || !grads->rgb ||
                        !grads->mean3d || !grads->cov3d || (with_feature && (!feats || !grads->feat))))
        return GS_ERR_ARG;
    if (with_feature &&
        (((uintptr_t)feats & 15) != 0 || ((uintptr_t)dL_dF & 15) != 0 || ((uintptr_t)grads->feat & 15) != 0))
        return GS_ERR_ARG;
    int st = ws_check(L, ws, ws_bytes);
    if (st) return st;
    if (n_gauss == 0) return GS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CamTable ct;
    make_camtable(cfg, cams, n_cams, ct);
    if (with_feature && !L.use_tiles) return GS_ERR_UNSUPPORTED;
    // Two independent chains: (h, re-walk, projection adjoint) on `stream`, the
    // feature-gradient reduction on the device's auxiliary stream, forked after the
    // work already queued on `stream` and joined back before returning.  The re-walk is
    // issue-bound and the reduction memory-bound, so they overlap.  On the CUDA-core block
    // product's path `stream` also waits (aux->hold) for the block records, so that the
    // product's CTAs are placed before the persistent re-walk's fill the SMs.
    std::unique_lock<std::mutex> lk(aux_mutex());
    const AuxStream *aux = with_feature ? aux_stream(s) : nullptr;
    if (aux) {
        if (cudaEventRecord(aux->fork, s) != cudaSuccess || cudaStreamWaitEvent(aux->s, aux->fork, 0) != cudaSuccess)
            return GS_ERR_CUDA;
    }
    bool ok = true;
    if (with_feature) {
        // h = dL/dF . f per slot: left in ws by gs_feature_blend_loss when the caller
        // says dL_dF is that call's and the call took the path that writes it
        const bool h_ready =
            (flags & GS_BWD_H_FROM_LOSS) && blend_loss_writes_h(cfg->feat_dtype, cfg->K, cfg->D, n_gauss);
        ok = launch_feature_grad(ct, L, cfg->feat_dtype, n_gauss, topk_idx, topk_w, dL_dF, grads->feat, ws,
                                 aux ? aux->s : s, aux ? s : nullptr, aux ? aux->hold : nullptr) &&
             (h_ready || launch_feature_h(L, cfg->feat_dtype, topk_idx, feats, dL_dF, ws, s));
    }
    ok = ok && launch_walk_bwd(ct, L, cfg->K, n_gauss, proj, ws, rgb_out, depth_out, topk_idx, topk_w, dL_dC, dL_dD,
                               with_feature, s);
    if (ok)
        launch_project_backward(ct, n_gauss, mean3d, cov3d, proj, ws_ptr<uint32_t>(ws, L.elem_off),
                                ws_ptr<uint32_t>(ws, L.elem_cnt), ws_ptr<float>(ws, L.inst_grad),
                                ws_ptr<uint8_t>(ws, L.inst_walked),
                                ws_ptr<float>(ws, L.elem_grad), ws_ptr<int>(ws, L.header), grads,
                                ws_ptr<float>(ws, L.pose_part), s);
    // the join is queued on every path after a fork, so a capture of `stream` stays whole
    if (aux) {
        if (cudaEventRecord(aux->join, aux->s) != cudaSuccess || cudaStreamWaitEvent(s, aux->join, 0) != cudaSuccess)
            return GS_ERR_CUDA;
    }
    if (!ok) return GS_ERR_UNSUPPORTED;
    return launch_status();
}

size_t gs_loss_scratch_size(int64_t n_pix)
{
    if (n_pix < 0) return 0;
    return sizeof(float) * (size_t)(n_pix + kSortBlocks + 64);
}

int gs_loss_cos_l1(const gs_config *cfg, int64_t n_pix, const void *F, const void *F_gt,
                   const float *rgb, const float *rgb_gt, const float *depth, const float *depth_gt,
                   float w_feat, float w_rgb, float w_depth,
                   void *dL_dF, float *dL_dC, float *dL_dD, float *loss,
                   void *scratch, size_t scratch_bytes, void *stream)
{
    if (!cfg_ok(cfg) || n_pix < 1) return GS_ERR_ARG;
    if (!F || !F_gt || !rgb || !rgb_gt || !depth || !depth_gt || !dL_dF || !dL_dC || !dL_dD || !loss)
        return GS_ERR_ARG;
    if (((uintptr_t)F & 15) || ((uintptr_t)F_gt & 15) || ((uintptr_t)dL_dF & 15)) return GS_ERR_ARG;
    if (!scratch || ((uintptr_t)scratch & 15) || scratch_bytes < gs_loss_scratch_size(n_pix)) return GS_ERR_WORKSPACE;
    launch_loss(cfg->feat_dtype, cfg->D, n_pix, F, F_gt, rgb, rgb_gt, depth, depth_gt, w_feat, w_rgb, w_depth, dL_dF,
                dL_dC, dL_dD, loss, (float *)scratch, (cudaStream_t)stream);
    return launch_status();
}

int gs_feature_blend_loss(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                          const int32_t *topk_idx, const float *topk_w, const void *feats, const void *F_gt,
                          const float *rgb, const float *rgb_gt, const float *depth, const float *depth_gt,
                          float w_feat, float w_rgb, float w_depth, void *F_out, void *dL_dF, float *dL_dC,
                          float *dL_dD, float *loss, void *ws, size_t ws_bytes, void *scratch, size_t scratch_bytes,
                          void *stream)
{
    WsLayout L;
    if (!make_layout(cfg, cams, n_cams, n_gauss, L)) return GS_ERR_ARG;
    if (!topk_idx || !topk_w || !F_gt || !rgb || !rgb_gt || !depth || !depth_gt || !F_out || !dL_dF || !dL_dC ||
        !dL_dD || !loss || (n_gauss > 0 && !feats))
        return GS_ERR_ARG;
    if (((uintptr_t)feats & 15) || ((uintptr_t)F_gt & 15) || ((uintptr_t)F_out & 15) || ((uintptr_t)dL_dF & 15))
        return GS_ERR_ARG;
    int st = ws_check(L, ws, ws_bytes);
    if (st) return st;
    if (!scratch || ((uintptr_t)scratch & 15) || scratch_bytes < gs_loss_scratch_size(L.P)) return GS_ERR_WORKSPACE;
    CamTable ct;
    make_camtable(cfg, cams, n_cams, ct);
    if (!launch_blend_loss(ct, cfg->feat_dtype, cfg->K, cfg->D, L.P, n_gauss, topk_idx, topk_w, feats, F_gt, rgb, rgb_gt, depth,
                           depth_gt, w_feat, w_rgb, w_depth, F_out, dL_dF, dL_dC, dL_dD, loss, (float *)scratch,
                           ws_ptr<float>(ws, L.hbuf), ws_ptr<int>(ws, L.header), (cudaStream_t)stream))
        return GS_ERR_UNSUPPORTED;
    return launch_status();
}

int gs_loss_geo_l1(int64_t n_pix, const float *rgb, const float *rgb_gt, const float *depth, const float *depth_gt,
                   float w_rgb, float w_depth, float *dL_dC, float *dL_dD, float *loss, void *scratch,
                   size_t scratch_bytes, void *stream)
{
    if (n_pix < 1 || !rgb || !rgb_gt || !depth || !depth_gt || !dL_dC || !dL_dD || !loss) return GS_ERR_ARG;
    if (!scratch || ((uintptr_t)scratch & 15) || scratch_bytes < gs_loss_scratch_size(n_pix)) return GS_ERR_WORKSPACE;
    launch_loss_geo(n_pix, rgb, rgb_gt, depth, depth_gt, w_rgb, w_depth, dL_dC, dL_dD, loss, (float *)scratch,
                    (cudaStream_t)stream);
    return launch_status();
}

int gs_adam_step(const gs_adam_tensor *tensors, int32_t n_tensors, int32_t step, float beta1, float beta2, float eps,
                 void *stream)
{
    if (n_tensors < 0 || n_tensors > GS_ADAM_MAX_TENSORS || step < 1) return GS_ERR_ARG;
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f)) return GS_ERR_ARG;
    if (n_tensors > 0 && !tensors) return GS_ERR_ARG;
    AdamTensor t[kAdamMaxTensors];
    int nt = 0;
    for (int i = 0; i < n_tensors; ++i) {
        const gs_adam_tensor &a = tensors[i];
        if (a.n < 0) return GS_ERR_ARG;
        if (a.n == 0) continue;
        if (!a.param || !a.grad || !a.exp_avg || !a.exp_avg_sq) return GS_ERR_ARG;
        if (((uintptr_t)a.param_bf16 & 7) != 0) return GS_ERR_ARG;
        t[nt++] = AdamTensor{a.param, a.grad, a.exp_avg, a.exp_avg_sq, (long long)a.n, a.lr,
                             (__nv_bfloat16 *)a.param_bf16};
    }
    if (nt == 0) return GS_OK;
    launch_adam(t, nt, step, beta1, beta2, eps, (cudaStream_t)stream);
    return launch_status();
}

int gs_feature_blend_vanilla(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss,
                             const float *proj, const void *feats, void *F_out, void *ws, size_t ws_bytes,
                             void *stream)
{
    WsLayout L;
    if (!make_layout(cfg, cams, n_cams, n_gauss, L)) return GS_ERR_ARG;
    if ((n_gauss > 0 && (!proj || !feats)) || (L.P > 0 && !F_out)) return GS_ERR_ARG;
    if (((uintptr_t)feats & 15) != 0 || ((uintptr_t)F_out & 15) != 0) return GS_ERR_ARG;
    int st = ws_check(L, ws, ws_bytes);
    if (st) return st;
    CamTable ct;
    make_camtable(cfg, cams, n_cams, ct);
    if (!launch_vanilla(cfg->feat_dtype, ct, L, n_gauss, proj, ws, feats, F_out, (cudaStream_t)stream))
        return GS_ERR_UNSUPPORTED;
    return launch_status();
}

int gs_prune_stats(const gs_config *cfg, const gs_camera *cams, int32_t n_cams, int32_t n_gauss, const float *proj,
                   const int32_t *topk_idx, void *ws, size_t ws_bytes, int32_t *topk_count, float *S, void *stream)
{
    WsLayout L;
    if (!make_layout(cfg, cams, n_cams, n_gauss, L)) return GS_ERR_ARG;
    if ((n_gauss > 0 && (!proj || !topk_count || !S)) || (L.PK > 0 && !topk_idx)) return GS_ERR_ARG;
    int st = ws_check(L, ws, ws_bytes);
    if (st) return st;
    CamTable ct;
    make_camtable(cfg, cams, n_cams, ct);
    if (!launch_prune_stats(ct, L, n_gauss, proj, topk_idx, ws, topk_count, S, (cudaStream_t)stream))
        return GS_ERR_UNSUPPORTED;
    return launch_status();
}

size_t gs_prune_select_workspace_size(int32_t n_gauss)
{
    if (n_gauss < 0) return 0;
    return prune_select_ws(n_gauss);
}

int gs_prune_select(int32_t n_gauss, const int32_t *topk_count, const float *S, int32_t tau, double ratio,
                    const float *expo, uint8_t *keep, void *ws, size_t ws_bytes, void *stream)
{
    if (n_gauss < 0 || !(ratio >= 0.0 && ratio <= 1.0)) return GS_ERR_ARG;
    if (n_gauss == 0) return GS_OK;
    if (!topk_count || !S || !expo || !keep) return GS_ERR_ARG;
    if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < prune_select_ws(n_gauss)) return GS_ERR_WORKSPACE;
    if (!launch_prune_select(n_gauss, topk_count, S, tau, ratio, expo, keep, ws, (cudaStream_t)stream))
        return GS_ERR_UNSUPPORTED;
    return launch_status();
}

int gs_set_wait_limit(void *ws, size_t ws_bytes, int64_t cycles, void *stream)
{
    if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < 256) return GS_ERR_WORKSPACE;
    const unsigned long long v = cycles > 0 ? (unsigned long long)cycles : 0ull;
    k_store_u64<<<1, 1, 0, (cudaStream_t)stream>>>(ws_ptr<unsigned long long>(ws, kHdrWaitLimitByte), v);
    return launch_status();
}

int gs_workspace_counts(const void *ws, size_t ws_bytes, void *stream, int64_t *n_instances,
                        int64_t *n_feature_rows)
{
    if (!ws || ws_bytes < 256) return GS_ERR_WORKSPACE;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GS_ERR_CUDA;
    uint32_t h[16];
    if (cudaMemcpy(h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return GS_ERR_CUDA;
    if (n_instances) *n_instances = (int64_t)h[1] + (int64_t)h[kHdrFresh];
    if (n_feature_rows) *n_feature_rows = (int64_t)h[8];
    return GS_OK;
}

int gs_binning_stats(const void *ws, size_t ws_bytes, void *stream, int64_t out[4])
{
    if (!ws || ws_bytes < 256) return GS_ERR_WORKSPACE;
    if (!out) return GS_ERR_ARG;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GS_ERR_CUDA;
    uint32_t h[16];
    if (cudaMemcpy(h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return GS_ERR_CUDA;
    out[0] = (int64_t)h[1] + (int64_t)h[kHdrFresh];
    out[1] = (int64_t)h[kHdrN1];
    out[2] = (int64_t)h[kHdrN2];
    out[3] = (int64_t)h[kHdrIncomplete];
    return GS_OK;
}

int gs_timer_enable(int on)
{
    Timers &t = timers();
    std::lock_guard<std::mutex> g(t.m);
    t.enabled = on != 0;
    for (bool &r : t.recorded) r = false;
    return GS_OK;
}

int gs_timer_read(int id, float *ms)
{
    if (id < 0 || id >= GS_TIMER_COUNT || !ms) return GS_ERR_ARG;
    Timers &t = timers();
    cudaEvent_t a, b;
    {
        std::lock_guard<std::mutex> g(t.m);
        if (!t.recorded[id]) return GS_ERR_ARG;
        a = t.ev[id][0];
        b = t.ev[id][1];
    }
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

int gs_sync_status(const void *ws, size_t ws_bytes, void *stream, int64_t *n_instances)
{
    if (!ws || ws_bytes < 256) return GS_ERR_WORKSPACE;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GS_ERR_CUDA;
    uint32_t h[16];
    if (cudaMemcpy(h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return GS_ERR_CUDA;
    if (n_instances) *n_instances = (int64_t)h[1] + (int64_t)h[kHdrFresh];
    if (h[0] & kErrOverflow) return GS_ERR_OVERFLOW;
    if (h[0] & kErrTimeout) return GS_ERR_TIMEOUT;
    return GS_OK;
}

}  // extern "C"
