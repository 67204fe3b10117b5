// lbp_decode / lbp_decode_host: launch planning for K_bp and K_osd.
//
// K_bp runs persistent: one CTA per SM, S groups of G threads per CTA, the
// graph image plus S shots' state in shared memory.  S and G come from the
// shared-memory budget, lbp_tune's stored shape or LBP_BP_SHAPE (read when
// the code was loaded, like every environment switch here); a call of
// at most one shot per SM that runs alone on the device gets one shot per CTA
// with up to 1024 threads.  K_osd follows on the same stream and drains the
// queue K_bp filled; no host round trip separates them.
//
// With OSD on, K_osd_warp (one warp per shot, sparse-aware; alone on the
// device with at most one shot per SM, its latency layout) drains the queue
// first; K_osd (one CTA per shot, dense) then takes the shots it handed over.
//
// Workspace (caller-owned device memory), 256-byte aligned sections:
//   counters   u32[64]  [0] next shot, [1] OSD queue length, [2] handed over
//   osd_list   u32[B]   shots handed to OSD            (osd only)
//   osd_llr    f32[B][n] their final lambda            (osd only)
//   overflow   u32[B]   queue positions K_osd_warp handed over (osd only)
//   osd_mat    u64[grid][m][ceil(n/64)] K_osd dense matrices (when they do
//                                                     not fit shared memory)
//   slots      u64[warps][C][ceil(n/64)] K_osd_warp dense-row pools
#include <algorithm>
#include <utility>
#include <vector>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include <cuda_fp16.h>

#include "bp_kernel.cuh"
#include "internal.h"
#include "launch.h"
#include "osd_dense_kernel.cuh"
#include "osd_kernel.cuh"
#include "osd_warp_kernel.cuh"
#include "timing.h"

namespace {

using namespace lbp;

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }
uint32_t align16u(uint32_t x) { return (x + 15u) & ~15u; }

int msg_bytes(int msg) { return msg == LBP_MSG_F32 ? 4 : (msg == LBP_MSG_F16 ? 2 : 1); }

// Index of the tuned launch shape kept per (check-node rule, message type).
int tuned_slot(int msg, int rule) {
    const int mi = msg >= 0 && msg < 3 ? msg : 0;
    return (rule == LBP_RULE_SUM_PRODUCT ? 3 : 0) + mi;
}

struct BpPlan {
    bool ell = false, graph_smem = true, state_smem = true, idx32 = false, surface = false, round = false;
    bool tab = false;            // index-image form with the bank-aware stride and pair table
    bool split = false;          // split state: ks message slots in shared memory, the rest in the workspace
    int ks = 0;
    uint32_t gbeta_bytes = 0;    // per-group workspace slice of a split state's other slots
    int groups = 0, G = 0, grid = 0;
    uint32_t state_bytes = 0, off_beta = 0, off_lam = 0, off_s = 0, off_shat = 0, off_misc = 0;
    size_t smem = 0;
};

struct OsdPlan {
    bool smem_mat = false;
    int grid = 0, n_pad = 1, wn = 0;
    uint32_t off_keys = 0, off_inv = 0, off_flags = 0, off_piv = 0, off_ebits = 0, off_mat = 0;
    size_t smem = 0;
};

struct OsdWarpPlan {
    bool ok = false;
    int warps = 0, grid = 0, C = 0, wn = 0;
    uint32_t image = 0, region = 0, off_keys = 0, off_tmp = 0, off_hist = 0, off_rflag = 0, off_pivk = 0,
             off_pivb = 0, off_saug = 0, off_x = 0, off_pcol = 0, off_prow = 0, off_pend = 0;
    uint32_t off_lb = 0, off_pool = 0;
    int Cs = 0;
    bool lat = false;
    size_t smem = 0;
};

struct WsLayout {
    size_t counters = 0, gstate = 0, osd_list = 0, osd_llr = 0, osd_mat = 0, overflow = 0, slots = 0,
           total = 0;
};

int validate_params(const lbp_params *p) {
    if (!p) return LBP_EINVAL;
    if (p->max_iter < 1 || p->max_iter > kMaxIter) return LBP_EINVAL;
    if (p->scale_mode != LBP_SCALE_CONST && p->scale_mode != LBP_SCALE_ADAPTIVE) return LBP_EINVAL;
    if (p->scale_mode == LBP_SCALE_CONST && !(p->scale_const > 0.0f && p->scale_const <= 1.0f)) return LBP_EINVAL;
    if (p->lottery != 0 && p->lottery != 1) return LBP_EINVAL;
    if (p->lottery_skip < 0) return LBP_EINVAL;
    if (p->osd != 0 && p->osd != 1) return LBP_EINVAL;
    if (p->msg != LBP_MSG_F32 && p->msg != LBP_MSG_F16 && p->msg != LBP_MSG_I8) return LBP_EINVAL;
    if (p->lottery_policy < LBP_LOTTERY_PROPOSED || p->lottery_policy > LBP_LOTTERY_PROPOSED_CURRENT) return LBP_EINVAL;
    if (p->rule != LBP_RULE_MIN_SUM && p->rule != LBP_RULE_SUM_PRODUCT) return LBP_EINVAL;
    if (p->reserved != 0) return LBP_EINVAL;
    return LBP_OK;
}

// Plan K_bp for this code and message type; returns LBP_ENOSYS if even one
// group does not fit in shared memory.
// Graph form of K_bp: 1 the index image, 2 the implicit Table III graph,
// 3 the round-periodic graph (one round's index table); the request, else
// LBP_GRAPH=table|implicit|round, else the tuned form, among the forms this
// code has; by default the index image, from shared memory where it fits
// beside one shot's state and from global memory otherwise.  Measured on
// GB300 the other two forms cost more instructions than the image's index
// loads save, even when the image is read from L2 (d=25 space-time code).
int graph_form(const lbp_code *c, int mi, int req_graph, size_t state_bytes) {
    auto ok = [&](int f) { return f == 1 || (f == 2 && c->surface) || (f == 3 && c->round); };
    if (req_graph >= 1 && req_graph <= 3) return ok(req_graph) ? req_graph : -1;
    if (c->env_graph == 1) return 1;
    if (c->env_graph >= 2 && ok(c->env_graph)) return c->env_graph;
    if (c->tuned_graph[mi] > 0 && ok(c->tuned_graph[mi])) return c->tuned_graph[mi];
    (void)state_bytes;
    return 1;
}

int plan_bp(const lbp_code *c, int msg, int rule, int64_t num_shots, BpPlan *out, int req_S = 0,
            int req_G = 0, int req_graph = 0, bool alone = true) {
    const int W32 = (c->m + 31) / 32;
    const int mi = tuned_slot(msg, rule);
    BpPlan p;
    // Bounded-degree ELL kernel when the code has an ELL image that fits.
    // Message rows: R = Mp + 2 words, or the bank-aware stride of the
    // index-image form (always in shared memory) when the code has one.
    auto state_layout = [&](int R, int slots = 0) {
        uint32_t o = 0;
        p.off_beta = o; o = align16u(o + static_cast<uint32_t>(msg_bytes(msg)) * (slots ? slots : c->ell.DC) * R);
        p.off_lam = o;  o = align16u(o + 4u * (c->ell.Np + 2));
        p.off_s = o;    o = align16u(o + 4u * W32);
        p.off_shat = o; o = align16u(o + 12u * W32);
        p.off_misc = o; o = align16u(o + 16u);
        p.state_bytes = o;
        return o;
    };
    uint32_t off = state_layout(c->ell.Mp + 2);
    size_t image = c->ell.bytes;
    const size_t budget0 = static_cast<size_t>(c->smem_optin);
    const int form = graph_form(c, mi, req_graph, off);
    if (form < 0) return LBP_ENOSYS;
    if (form == 1 && c->tab_R > 0) {
        off = state_layout(c->tab_R);
        p.tab = true;
    }
    if (form == 2 || form == 3) {
        // Implicit or round-periodic graph: the state and at most a small
        // round image in shared memory.
        const size_t rimg = form == 3 ? c->rnd.bytes : 0;
        const size_t budget_s = budget0 > rimg ? budget0 - rimg : 0;
        p.ell = true;
        p.surface = form == 2;
        p.round = form == 3;
        p.graph_smem = form == 3;
        p.state_smem = off <= budget_s;
        int S = 1, G = 1024;
        if (p.state_smem) {
            const int S_fit = static_cast<int>(budget_s / off);
            if (S_fit >= 6) { G = 96; S = S_fit < 10 ? S_fit : 10; }
            else if (S_fit >= 4) { G = 256; S = 4; }
            else if (S_fit >= 2) { G = 512; S = 2; }
            if (c->tuned_G[mi] > 0 && c->tuned_graph[mi] == form) {
                G = c->tuned_G[mi];
                S = c->tuned_groups[mi] < S_fit ? c->tuned_groups[mi] : S_fit;
            }
            int s_req = req_S, g_req = req_G;
            if (!g_req) {
                s_req = c->env_S;
                g_req = c->env_G;
            }
            if (g_req == 64 || g_req == 96 || g_req == 128 || g_req == 192 || g_req == 256 || g_req == 512 ||
                g_req == 1024) {
                G = g_req;
                S = s_req > 0 && s_req < S_fit ? s_req : S_fit;
            } else if (num_shots <= c->sm_count) {
                S = 1;              // a batch that does not fill the GPU: one shot per CTA
                G = 256;
            }
            if (S * G > 1024) S = 1024 / G;
            if (G > 32 && S > 15) S = 15;
        } else {
            G = req_G == 1024 ? 1024 : 512;
            S = 1024 / G;
        }
        if (S < 1) S = 1;
        p.groups = S;
        p.G = G;
        p.smem = rimg + (p.state_smem ? static_cast<size_t>(S) * off : static_cast<size_t>(16) * S);
        const int64_t need = (num_shots + S - 1) / S;
        p.grid = static_cast<int>(need < c->sm_count ? need : c->sm_count);
        if (p.grid < 1) p.grid = 1;
        *out = p;
        return LBP_OK;
    }
    p.ell = c->d_ell != nullptr;
    p.idx32 = p.ell && c->ell.idx_bytes == 4;
    if (p.ell && (p.idx32 || image + off > budget0)) {
        // Large code: graph image from global memory (L2); state in shared
        // memory when one group's fits, else in the workspace.
        p.graph_smem = false;
        p.state_smem = off <= budget0;
        // The requested shape, else LBP_BP_SHAPE, else lbp_tune's stored one.
        if (!req_G && c->env_G) {
            req_S = c->env_S;
            req_G = c->env_G;
        }
        if (!req_G && c->tuned_G[mi] > 0 && c->tuned_graph[mi] == 1) {
            req_S = c->tuned_groups[mi];
            req_G = c->tuned_G[mi];
        }
        // Split state: when one shot's state does not fit, all message slots
        // but the last two stay in shared memory with the posteriors and
        // syndrome words, if they fit (one shot per CTA of 512, 768 or 1024
        // threads: the tuned or requested width, else 1024); the last two
        // slots go to a per-group workspace slice.  A request for several groups
        // (S > 1) or for 256 threads keeps the whole state in the workspace.
        const int s_eff = req_G > 0 ? std::min(req_S > 0 ? req_S : 1, 1024 / req_G) : 1;
        const bool split_req = req_G == 0 || (s_eff <= 1 && (req_G == 512 || req_G == 768 || req_G == 1024));
        if (!p.state_smem && !p.idx32 && split_req) {
            const int ks = c->ell.DC - 2;            // the last two slots go to the workspace
            {
                const uint32_t o = state_layout(c->ell.Mp + 2, ks);
                if (o <= budget0) {
                    p.split = true;
                    p.ks = ks;
                    p.gbeta_bytes = static_cast<uint32_t>(
                        align256(static_cast<size_t>(msg_bytes(msg)) * (c->ell.DC - ks) * (c->ell.Mp + 2)));
                    p.state_smem = true;
                    p.groups = 1;
                    p.G = 1024;
                    if (req_G == 512 || req_G == 768) p.G = req_G;
                    p.smem = o;
                    const int64_t need = num_shots;
                    p.grid = static_cast<int>(need < c->sm_count ? need : c->sm_count);
                    if (p.grid < 1) p.grid = 1;
                    *out = p;
                    return LBP_OK;
                }
            }
            off = state_layout(c->ell.Mp + 2);
        }
        int G = 1024, S = 1;
        if (p.state_smem) {
            S = static_cast<int>(budget0 / off);
            if (S < 1) S = 1;
            G = 1024 / S >= 1024 ? 1024 : (1024 / S >= 512 ? 512 : 256);
            if (S * G > 1024) S = 1024 / G;
        } else {
            G = 512;
            S = 2;
        }
        if (p.idx32) {
            // 32-bit images have one shape per placement.
            if (p.state_smem) { G = 1024; S = 1; } else { G = 512; S = 2; }
        } else if (req_G == 256 || req_G == 512 || req_G == 1024) {
            G = req_G;
            if (req_S > 0) S = req_S;
            if (p.state_smem && static_cast<size_t>(S) * off > budget0) S = static_cast<int>(budget0 / off);
            if (S * G > 1024) S = 1024 / G;
            if (S < 1) S = 1;
        }
        p.groups = S;
        p.G = G;
        p.smem = p.state_smem ? static_cast<size_t>(S) * off : static_cast<size_t>(16) * S;
        const int64_t need = (num_shots + S - 1) / S;
        p.grid = static_cast<int>(need < c->sm_count ? need : c->sm_count);
        if (p.grid < 1) p.grid = 1;
        *out = p;
        return LBP_OK;
    }
    if (!p.ell) {
        if (!c->d_image) return LBP_ENOSYS;
        off = 0;
        p.off_beta = off; off = align16u(off + static_cast<uint32_t>(msg_bytes(msg)) * c->nnz);
        p.off_lam = off;  off = align16u(off + 4u * c->n);
        p.off_s = off;    off = align16u(off + 4u * W32);
        p.off_shat = off; off = align16u(off + 12u * W32);
        p.off_misc = off; off = align16u(off + 16u);
        p.state_bytes = off;
        image = c->img.bytes;
    }
    const size_t budget = static_cast<size_t>(c->smem_optin);
    if (image + static_cast<size_t>(p.state_bytes) > budget) return LBP_ENOSYS;
    const int S_fit = static_cast<int>((budget - image) / p.state_bytes);
    int S = S_fit;
    // Default shape: threads per group scale with the code (at most 128; 96
    // when the ELL kernel has room for at least 6 groups, which balances the
    // d=11 space-time code best); lbp_tune replaces it by measurement.
    int G = 32;
    while (G < 128 && G * 2 <= 1024 / (S > 0 ? S : 1) && (G < c->m / 4 || G < c->n / 16)) G *= 2;
    if (p.ell && G == 128 && S_fit >= 6) G = 96;
    if (c->tuned_G[mi] > 0 && c->tuned_graph[mi] == 1) {
        G = c->tuned_G[mi];
        S = c->tuned_groups[mi] < S_fit ? c->tuned_groups[mi] : S_fit;
    }
    // Explicit shape (lbp_tune candidates), then the LBP_BP_SHAPE override "S,G".
    int s_req = req_S, g_req = req_G;
    if (!g_req) {
        s_req = c->env_S;
        g_req = c->env_G;
    }
    const bool g_ok = g_req == 32 || g_req == 64 || g_req == 96 || g_req == 128 || g_req == 192 ||
                      g_req == 256 || (p.ell && (g_req == 512 || g_req == 1024));
    if (s_req > 0 && g_ok) {
        G = g_req;
        S = s_req < S_fit ? s_req : S_fit;
    } else if (num_shots <= c->sm_count) {
        // A batch that does not fill the GPU: one shot per CTA, for the
        // lowest latency (the SMs would idle anyway).  Alone on the device,
        // the ELL kernel gets a thread per column pair, up to 1024: at this
        // size an iteration's time is the latency of its dependent steps,
        // not its instructions.
        S = 1;
        G = 256;
        while (alone && p.ell && G < 1024 && G < (c->ell.Np + 1) / 2) G *= 2;
    }
    if (!p.ell && G != 32 && G != 64 && G != 128 && G != 256) G = 128;
    if (S * G > 1024) S = 1024 / G;
    if (G > 32 && S > 15) S = 15;     // named barriers 1..15
    if (S < 1) S = 1;
    p.groups = S;
    p.G = G;
    p.smem = image + static_cast<size_t>(S) * p.state_bytes;
    const int64_t need = (num_shots + S - 1) / S;
    p.grid = static_cast<int>(need < c->sm_count ? need : c->sm_count);
    if (p.grid < 1) p.grid = 1;
    *out = p;
    return LBP_OK;
}

int plan_osd(const lbp_code *c, int64_t num_shots, OsdPlan *out) {
    OsdPlan p;
    p.wn = (c->n + 63) / 64;
    while (p.n_pad < c->n) p.n_pad <<= 1;
    uint32_t off = 0;
    p.off_keys = off;  off = align16u(off + 8u * p.n_pad);
    p.off_inv = off;   off = align16u(off + 4u * c->n);
    p.off_flags = off; off = align16u(off + 3u * c->m);
    p.off_piv = off;   off = align16u(off + 4u * (4 + 2 * c->m));
    p.off_ebits = off; off = align16u(off + 8u * p.wn);
    p.off_mat = off;
    const size_t mat = 8ull * c->m * p.wn;
    if (off > static_cast<size_t>(c->smem_optin)) return LBP_ENOSYS;
    p.smem_mat = off + mat <= static_cast<size_t>(c->smem_optin);
    p.smem = p.smem_mat ? off + mat : off;
    const int64_t g = num_shots < c->sm_count ? num_shots : c->sm_count;
    p.grid = static_cast<int>(g < 1 ? 1 : g);
    *out = p;
    return LBP_OK;
}

// K_osd_warp plan: CSR prefix of the 16-bit image, then one region per warp.
constexpr int kOsdMaxWarps = 24;

void plan_osd_warp(const lbp_code *c, int64_t num_shots, OsdWarpPlan *out) {
    OsdWarpPlan p;
    if (!c->d_image || c->m < 1 || c->n < 1) { *out = p; return; }
    p.wn = (c->n + 63) / 64;
    const int W32 = (c->m + 31) / 32;
    uint32_t off = 0;
    p.off_keys = off;  off = align16u(off + 8u * c->m);
    // Only the keys and the radix sort's buffer and digit histogram are live
    // during the sort; the elimination's arrays, first written after it,
    // share their bytes.
    const uint32_t u0 = off;
    p.off_tmp = u0;
    p.off_hist = u0 + align16u(8u * c->m);
    const uint32_t sort_end = p.off_hist + 4u * 256;
    p.off_pcol = off;  off = align16u(off + 2u * c->m);
    p.off_prow = off;  off = align16u(off + 2u * c->m);
    p.off_rflag = off; off = align16u(off + 2u * c->m);
    p.off_pivb = off;  off = align16u(off + 4u * W32);
    p.off_saug = off;  off = align16u(off + 4u * W32);
    p.off_pend = off;
    // The solution bits X [wn] and the column -> pivot index map [n], both
    // built after the elimination, share the dead keys' bytes when they fit.
    const uint32_t xb = align16u(8u * static_cast<uint32_t>(p.wn));
    const bool in_keys = xb + 2u * static_cast<uint32_t>(c->n) <= 8u * static_cast<uint32_t>(c->m);
    // End of the arrays live during the sort or the elimination.
    auto live_end = [&](int C) -> uint32_t {
        const uint32_t end = align16u(p.off_pend + 8u * static_cast<uint32_t>(C));
        return end > align16u(sort_end) ? end : align16u(sort_end);
    };
    auto region_for = [&](int C) -> uint32_t {
        const uint32_t end = live_end(C);
        return in_keys ? end : align16u(end + xb + 2u * static_cast<uint32_t>(c->n));
    };
    p.image = c->img.off_col_ptr;             // row_ptr and col_idx only
    const size_t budget = static_cast<size_t>(c->smem_optin) - p.image;
    auto warps_for = [&](int C) {
        const size_t w = budget / region_for(C);
        return static_cast<int>(w < kOsdMaxWarps ? w : kOsdMaxWarps);
    };
    // Pool rows C (changed rows a shot may hold before it is handed to
    // K_osd): half of m, at least 192, with the pool at most 1 GiB of
    // workspace; LBP_OSD_POOL_ROWS overrides.  Codes whose elimination
    // changes many rows (the unrotated d=11 space-time code needs ~450 at
    // p = 0.003) would otherwise send a quarter of their OSD shots to K_osd.
    int C = c->m / 2 > 192 ? c->m / 2 : 192;
    if (C > c->m) C = c->m;
    if (c->env_pool_rows > 0) {
        if (c->env_pool_rows <= c->m) C = c->env_pool_rows;
    } else if (warps_for(C) >= 1) {
        const int floor_c = c->m < 192 ? c->m : 192;
        // Up to 15% fewer rows when that fits another warp per SM (the
        // kernel is latency-bound, so warps are throughput).
        const int w0 = warps_for(C);
        for (int c2 = C - 1; c2 >= floor_c && c2 * 20 >= C * 17; --c2) {
            if (warps_for(c2) > w0) {
                C = c2;
                break;
            }
        }
        const size_t per_row = static_cast<size_t>(c->sm_count) * warps_for(C) * p.wn * 8u;
        const size_t cap = (static_cast<size_t>(1) << 30) / per_row;
        if (static_cast<size_t>(C) > cap) C = cap > static_cast<size_t>(floor_c) ? static_cast<int>(cap) : floor_c;
    }
    p.C = C;
    p.region = region_for(C);
    p.off_x = in_keys ? p.off_keys : live_end(C);
    p.off_pivk = p.off_x + xb;
    if (static_cast<size_t>(p.region) * 2 > budget) { *out = p; return; }
    p.warps = warps_for(C);
    p.smem = p.image + static_cast<size_t>(p.warps) * p.region;
    const int64_t need = (num_shots + p.warps - 1) / p.warps;
    p.grid = static_cast<int>(need < c->sm_count ? need : c->sm_count);
    if (p.grid < 1) p.grid = 1;
    p.ok = true;
    *out = p;
}

// Latency layout of K_osd_warp, for a batch of at most one shot per SM: one
// warp per CTA, whose region also holds lambda's order bits [n] and the first
// Cs rows of the dense-row pool (as many as fit, at most C); the pool keeps
// the throughput layout's C rows, the rest in the workspace, so no more shots
// overflow to K_osd.  LBP_OSD_LAT=0 turns it off.
bool plan_osd_lat(const lbp_code *c, int64_t num_shots, const OsdWarpPlan &wp, OsdWarpPlan *out) {
    if (!wp.ok || num_shots > c->sm_count) return false;
    if (!c->env_osd_lat) return false;
    OsdWarpPlan p = wp;
    const size_t budget = static_cast<size_t>(c->smem_optin) - p.image;
    const uint32_t lbb = align16u(4u * static_cast<uint32_t>(c->n));
    p.off_lb = p.region;                       // after pend [C], as in the throughput layout
    p.off_pool = align16u(p.off_lb + lbb);
    if (budget < static_cast<size_t>(p.off_pool) + 8u * static_cast<size_t>(p.wn)) return false;
    size_t Cs = (budget - p.off_pool) / (8u * static_cast<size_t>(p.wn));
    if (Cs > static_cast<size_t>(p.C)) Cs = static_cast<size_t>(p.C);
    p.Cs = static_cast<int>(Cs);
    p.region = align16u(p.off_pool + 8u * static_cast<uint32_t>(p.Cs) * static_cast<uint32_t>(p.wn));
    p.warps = 1;
    p.smem = static_cast<size_t>(p.image) + p.region;
    if (p.smem > static_cast<size_t>(c->smem_optin)) return false;
    const int64_t g = num_shots < c->sm_count ? num_shots : c->sm_count;
    p.grid = static_cast<int>(g < 1 ? 1 : g);
    p.lat = true;
    *out = p;
    return true;
}

WsLayout layout(const lbp_code *c, const lbp_params *prm, int64_t num_shots, const OsdPlan *op,
                const OsdWarpPlan *wp, const BpPlan *bp) {
    WsLayout w;
    size_t off = 0;
    w.counters = off; off = align256(off + 256);
    if (bp && (!bp->state_smem || bp->split)) {
        // Sized for every launch shape (at most 1024 / 256 groups per CTA, one
        // CTA per SM), so lbp_tune's candidates and any tuned shape fit; a
        // split state (one group per CTA in every shape) needs the slice of
        // its workspace slots per CTA.
        w.gstate = off;
        const size_t slice = bp->split ? bp->gbeta_bytes : bp->state_bytes;
        off = align256(off + static_cast<size_t>(c->sm_count) * (bp->split ? 1 : 4) * slice);
    }
    if (prm->osd) {
        w.osd_list = off; off = align256(off + 4ull * num_shots);
        w.osd_llr = off;  off = align256(off + 4ull * num_shots * c->n);
        w.overflow = off; off = align256(off + 4ull * num_shots);
        if (op && !op->smem_mat) {
            w.osd_mat = off;
            off = align256(off + 8ull * op->grid * c->m * op->wn);
        }
        if (wp && wp->ok) {
            const size_t warps = static_cast<size_t>(wp->grid) * wp->warps;
            w.slots = off; off = align256(off + 8ull * warps * wp->C * wp->wn);
        }
    }
    w.total = off;
    return w;
}

template <typename K>
int set_smem(K kernel, size_t bytes) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(bytes)) != cudaSuccess) {
        cudaGetLastError();
        return LBP_ECUDA;
    }
    return LBP_OK;
}

template <typename MsgT, int G>
int launch_bp_g(const BpPlan &p, const BpArgs &a, cudaStream_t s) {
    auto k = bp_kernel<MsgT, G>;
    int rc = set_smem(k, p.smem);
    if (rc) return rc;
    k<<<p.grid, p.groups * G, p.smem, s>>>(a);
    return LBP_OK;
}

template <typename MsgT>
int launch_bp_t(const BpPlan &p, const BpArgs &a, cudaStream_t s) {
    switch (p.G) {
        case 32: return launch_bp_g<MsgT, 32>(p, a, s);
        case 64: return launch_bp_g<MsgT, 64>(p, a, s);
        case 128: return launch_bp_g<MsgT, 128>(p, a, s);
        case 256: return launch_bp_g<MsgT, 256>(p, a, s);
        default: return LBP_ENOSYS;
    }
}

int check_launch() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBP_OK : LBP_ECUDA;
}

// K_osd_warp then K_osd on the OSD queue that K_bp filled (counters[1]
// shots in osd_list / osd_llr), for one code: shared by lbp_decode and by
// each item of a merged launch.
int launch_osd(const lbp_code *c, int64_t B, const uint64_t *syn, uint64_t *err, uint8_t *osd_out,
               unsigned int *counters, uint8_t *base, const WsLayout &w, const OsdPlan &op, OsdWarpPlan wp,
               uint32_t *osd_list, float *osd_llr, cudaStream_t stream, bool alone) {
    int rc = LBP_OK;
    if (c->osd_dense) {
        // Small code: K_osd_dense solves every queued shot (no pool, no
        // hand-over to K_osd).
        OsdDenseArgs d;
        std::memset(&d, 0, sizeof(d));
        d.image = c->d_image;
        d.img = c->img;
        d.image_bytes = c->img.off_col_ptr;       // row_ptr and col_idx only
        d.m = c->m; d.n = c->n; d.wn = (c->n + 63) / 64; d.rank = c->osd_rank;
        d.syn = syn; d.err = err; d.osd_out = osd_out;
        d.counters = counters;
        d.osd_list = osd_list; d.osd_llr = osd_llr;
        d.off_perm = align16u(4u * static_cast<uint32_t>(c->n));
        d.off_x = d.off_perm + align16u(2u * static_cast<uint32_t>(c->n));
        d.region_bytes = d.off_x + align16u(8u * static_cast<uint32_t>(d.wn));
        const int64_t need = (B + kOsdDenseWarps - 1) / kOsdDenseWarps;
        const int64_t cap = 2 * static_cast<int64_t>(c->sm_count);
        const int grid = static_cast<int>(need < 1 ? 1 : (need < cap ? need : cap));
        const size_t smem = d.image_bytes + static_cast<size_t>(kOsdDenseWarps) * d.region_bytes;
        void *td = timing_begin(stream);
        rc = launch_osd_dense(d, c->osd_RL, c->osd_WN, grid, smem, stream);
        timing_end(td, stream, kTimeOsd);
        return rc;
    }
    if (wp.ok) {
        OsdWarpPlan lp;
        if (alone && plan_osd_lat(c, B, wp, &lp)) wp = lp;
        OsdWarpArgs ow;
        std::memset(&ow, 0, sizeof(ow));
        ow.image = c->d_image;
        ow.img = c->img;
        ow.m = c->m; ow.n = c->n; ow.wn = wp.wn; ow.C = wp.C;
        ow.syn = syn; ow.err = err; ow.osd_out = osd_out;
        ow.counters = counters;
        ow.osd_list = osd_list; ow.osd_llr = osd_llr;
        ow.overflow = reinterpret_cast<uint32_t *>(base + w.overflow);
        ow.slots = reinterpret_cast<uint64_t *>(base + w.slots);
        ow.image_bytes = wp.image;
        ow.region_bytes = wp.region;
        ow.off_keys = wp.off_keys; ow.off_rflag = wp.off_rflag; ow.off_pivk = wp.off_pivk;
        ow.off_tmp = wp.off_tmp; ow.off_hist = wp.off_hist;
        ow.off_pivb = wp.off_pivb; ow.off_saug = wp.off_saug; ow.off_x = wp.off_x;
        ow.off_pcol = wp.off_pcol; ow.off_prow = wp.off_prow; ow.off_pend = wp.off_pend;
        ow.off_lb = wp.off_lb; ow.off_pool = wp.off_pool; ow.Cs = wp.Cs;
        rc = wp.lat ? set_smem(osd_warp_kernel<1, true>, wp.smem)
                    : set_smem(osd_warp_kernel<kOsdMaxWarps, false>, wp.smem);
        if (rc) return rc;
        void *tw = timing_begin(stream);
        if (wp.lat) {
            osd_warp_kernel<1, true><<<wp.grid, 32, wp.smem, stream>>>(ow);
        } else {
            osd_warp_kernel<kOsdMaxWarps, false><<<wp.grid, wp.warps * 32, wp.smem, stream>>>(ow);
        }
        timing_end(tw, stream, kTimeOsd);
        rc = check_launch();
        if (rc) return rc;
    }
    OsdArgs o;
    std::memset(&o, 0, sizeof(o));
    o.m = c->m; o.n = c->n;
    o.row_ptr = c->d_row_ptr; o.col_idx = c->d_col_idx;
    o.syn = syn; o.err = err; o.osd_out = osd_out;
    o.counters = counters;
    o.count_slot = wp.ok ? 2 : 1;
    o.qmap = wp.ok ? reinterpret_cast<const uint32_t *>(base + w.overflow) : nullptr;
    o.osd_list = osd_list; o.osd_llr = osd_llr;
    o.gmat = op.smem_mat ? nullptr : reinterpret_cast<uint64_t *>(base + w.osd_mat);
    o.n_pad = op.n_pad; o.wn = op.wn;
    o.off_keys = op.off_keys; o.off_inv = op.off_inv; o.off_flags = op.off_flags;
    o.off_piv = op.off_piv; o.off_ebits = op.off_ebits; o.off_mat = op.off_mat;
    rc = set_smem(op.smem_mat ? osd_kernel<true> : osd_kernel<false>, op.smem);
    if (rc) return rc;
    void *to = timing_begin(stream);
    if (op.smem_mat) {
        osd_kernel<true><<<op.grid, 1024, op.smem, stream>>>(o);
    } else {
        osd_kernel<false><<<op.grid, 1024, op.smem, stream>>>(o);
    }
    timing_end(to, stream, kTimeOsd);
    rc = check_launch();
    return rc;
}

}  // namespace

namespace lbp {

int decode_device(const lbp_code *c, const lbp_params *prm, int64_t B, const uint64_t *syn,
                  uint64_t *err, uint8_t *conv, uint8_t *osd_out, int32_t *iters, float *llr,
                  void *ws, size_t ws_bytes, cudaStream_t stream, bool alone) {
    return decode_device_shaped(c, prm, B, syn, err, conv, osd_out, iters, llr, ws, ws_bytes, stream,
                                0, 0, nullptr, 0, alone);
}

int decode_device_shaped(const lbp_code *c, const lbp_params *prm, int64_t B, const uint64_t *syn,
                         uint64_t *err, uint8_t *conv, uint8_t *osd_out, int32_t *iters, float *llr,
                         void *ws, size_t ws_bytes, cudaStream_t stream, int req_S, int req_G,
                         float *bp_ms, int req_graph, bool alone) {
    BpPlan bp;
    int rc = plan_bp(c, prm->msg, prm->rule, B, &bp, req_S, req_G, req_graph, alone);
    if (rc) return rc;
    // The lottery ablation (U from this iteration's s_hat) is built into the
    // index-image form in shared memory and the general kernel only.
    if (prm->lottery_policy == LBP_LOTTERY_PROPOSED_CURRENT && bp.ell &&
        !(bp.graph_smem && !bp.surface && !bp.round))
        return LBP_ENOSYS;
    OsdPlan op;
    OsdWarpPlan wp;
    if (prm->osd) {
        rc = plan_osd(c, B, &op);
        if (rc) return rc;
        plan_osd_warp(c, B, &wp);
    }
    const WsLayout w = layout(c, prm, B, prm->osd ? &op : nullptr, prm->osd ? &wp : nullptr, &bp);
    if (!ws || ws_bytes < w.total) return LBP_ENOMEM;
    if (reinterpret_cast<uintptr_t>(ws) & 255u) return LBP_EINVAL;
    uint8_t *base = static_cast<uint8_t *>(ws);
    unsigned int *counters = reinterpret_cast<unsigned int *>(base + w.counters);
    if (cudaMemsetAsync(counters, 0, 256, stream) != cudaSuccess) { cudaGetLastError(); return LBP_ECUDA; }

    BpArgs a;
    std::memset(&a, 0, sizeof(a));
    a.image = c->d_image;
    a.img = c->img;
    a.m = c->m; a.n = c->n;
    a.max_iter = prm->max_iter; a.scale_mode = prm->scale_mode; a.scale_const = prm->scale_const;
    a.lottery = prm->lottery; a.lottery_skip = prm->lottery_skip; a.osd = prm->osd;
    a.policy = prm->lottery_policy;
    a.rule = prm->rule;
    a.seed = prm->seed; a.shot_offset = prm->shot_offset;
    a.num_shots = B;
    a.syn = syn; a.err = err; a.conv = conv; a.osd_out = osd_out; a.iters = iters; a.llr = llr;
    a.counters = counters;
    a.osd_list = prm->osd ? reinterpret_cast<uint32_t *>(base + w.osd_list) : nullptr;
    a.osd_llr = prm->osd ? reinterpret_cast<float *>(base + w.osd_llr) : nullptr;
    a.state_bytes = bp.state_bytes;
    a.off_beta = bp.off_beta; a.off_lam = bp.off_lam; a.off_s = bp.off_s;
    a.off_shat = bp.off_shat; a.off_misc = bp.off_misc;
    void *tk = timing_begin(stream);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (bp_ms) {
        if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) {
            cudaGetLastError();
            return LBP_ECUDA;
        }
        cudaEventRecord(t0, stream);
    }
    if (bp.ell) {
        BpEllArgs e;
        std::memset(&e, 0, sizeof(e));
        e.image = c->d_ell;
        e.img = c->ell;
        e.m = a.m; e.n = a.n; e.max_iter = a.max_iter; e.scale_mode = a.scale_mode;
        e.scale_const = a.scale_const; e.lottery = a.lottery; e.lottery_skip = a.lottery_skip;
        e.osd = a.osd; e.seed = a.seed; e.shot_offset = a.shot_offset; e.num_shots = a.num_shots;
        e.policy = a.policy;
        e.rule = a.rule;
        e.syn = a.syn; e.err = a.err; e.conv = a.conv; e.osd_out = a.osd_out; e.iters = a.iters;
        e.llr = a.llr; e.counters = a.counters; e.osd_list = a.osd_list; e.osd_llr = a.osd_llr;
        e.state_bytes = a.state_bytes; e.off_beta = a.off_beta; e.off_lam = a.off_lam;
        e.off_s = a.off_s; e.off_shat = a.off_shat; e.off_misc = a.off_misc;
        e.gstate = (bp.state_smem && !bp.split) ? nullptr : base + w.gstate;
        e.gbeta_bytes = bp.gbeta_bytes;
        const int R = bp.tab ? c->tab_R : c->ell.Mp + 2;
        e.magic = static_cast<uint32_t>((1ull << 32) / static_cast<uint64_t>(R) + 1);
        e.tab_R = bp.tab ? c->tab_R : 0;
        e.off_ptab = bp.tab ? c->tab_off_ptab : 0u;
        e.surf = c->surf;
        e.rnd = c->rnd;
        e.mu_tab = c->d_mu_pad;
        if (bp.round) {
            e.image = c->d_round;                         // staged instead of the index image
            e.img.bytes = c->rnd.bytes;
        }
        const LaunchShape shp{bp.grid, bp.groups, bp.G, bp.smem, bp.graph_smem, bp.state_smem, bp.idx32,
                              bp.surface, bp.round, bp.split, false};
        const bool sp = prm->rule == LBP_RULE_SUM_PRODUCT;
        switch (prm->msg) {
            case LBP_MSG_F32:
                rc = (sp ? launch_bp_ell_sp_f32 : launch_bp_ell_f32)(shp, e, c->ell.DC, c->ell.DV, stream);
                break;
            case LBP_MSG_F16:
                rc = (sp ? launch_bp_ell_sp_f16 : launch_bp_ell_f16)(shp, e, c->ell.DC, c->ell.DV, stream);
                break;
            default:
                rc = (sp ? launch_bp_ell_sp_i8 : launch_bp_ell_i8)(shp, e, c->ell.DC, c->ell.DV, stream);
                break;
        }
    } else {
        switch (prm->msg) {
            case LBP_MSG_F32: rc = launch_bp_t<float>(bp, a, stream); break;
            case LBP_MSG_F16: rc = launch_bp_t<__half>(bp, a, stream); break;
            default: rc = launch_bp_t<int8_t>(bp, a, stream); break;
        }
    }
    timing_end(tk, stream, kTimeBp);
    if (bp_ms) {
        cudaEventRecord(t1, stream);
        cudaEventSynchronize(t1);
        if (cudaEventElapsedTime(bp_ms, t0, t1) != cudaSuccess) *bp_ms = -1.0f;
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
    }
    if (rc) return rc;
    rc = check_launch();
    if (rc) return rc;
    if (prm->osd) rc = launch_osd(c, B, syn, err, osd_out, counters, base, w, op, wp,
                                  a.osd_list, a.osd_llr, stream, alone);
    return rc;
}

}  // namespace lbp

namespace {

int check_common(const lbp_code *c, const lbp_params *prm, int64_t B) {
    if (!c) return LBP_EINVAL;
    int rc = validate_params(prm);
    if (rc) return rc;
    if (B < 0 || B > (1ll << 31)) return LBP_EINVAL;
    return LBP_OK;
}

}  // namespace

extern "C" size_t lbp_workspace_size(const lbp_code *code, const lbp_params *params, int64_t num_shots) {
    if (check_common(code, params, num_shots)) return 0;
    OsdPlan op;
    OsdWarpPlan wp;
    if (params->osd) {
        if (plan_osd(code, num_shots, &op)) return 0;
        plan_osd_warp(code, num_shots, &wp);
    }
    BpPlan bp;
    if (plan_bp(code, params->msg, params->rule, num_shots, &bp)) return 0;
    return layout(code, params, num_shots, params->osd ? &op : nullptr, params->osd ? &wp : nullptr, &bp).total;
}

extern "C" int lbp_decode(const lbp_code *code, const lbp_params *params, int64_t num_shots,
                          const uint64_t *syndromes, uint64_t *err_out, uint8_t *converged,
                          uint8_t *osd_out, int32_t *iters_out, float *llr_out,
                          void *workspace, size_t workspace_bytes, void *stream) {
    int rc = check_common(code, params, num_shots);
    if (rc) return rc;
    if (num_shots == 0) return LBP_OK;
    if (!syndromes || !err_out || !converged || !iters_out) return LBP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != code->device) return LBP_EINVAL;
    return decode_device(code, params, num_shots, syndromes, err_out, converged, osd_out, iters_out,
                         llr_out, workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
}

namespace {

// lbp_decode_host pipelines calls of at least 2 * kHostChunkShots shots.
constexpr int64_t kHostChunkShots = 131072;

// The two copy streams of lbp_decode_host's pipeline, per device, created on
// first use and kept for the life of the process.
struct CopyStreams {
    cudaStream_t in = nullptr, out = nullptr;
};

bool copy_streams(int dev, CopyStreams *out) {
    static std::mutex mu;
    static CopyStreams per_dev[64];
    if (dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lk(mu);
    CopyStreams &c = per_dev[dev];
    if (!c.in) {
        cudaStream_t a = nullptr, b = nullptr;
        if (cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            if (a) cudaStreamDestroy(a);
            return false;
        }
        c.in = a;
        c.out = b;
    }
    *out = c;
    return true;
}

struct HostStage {
    size_t syn, err, conv, osd, iters, decode_ws, total, llr, total_llr;
};

HostStage host_stage(const lbp_code *c, const lbp_params *prm, int64_t B) {
    HostStage h;
    const size_t wm = (c->m + 63) / 64, wn = (c->n + 63) / 64;
    size_t off = 0;
    h.syn = off;   off = align256(off + 8ull * wm * B);
    h.err = off;   off = align256(off + 8ull * wn * B);
    h.conv = off;  off = align256(off + static_cast<size_t>(B));
    h.osd = off;   off = align256(off + static_cast<size_t>(B));
    h.iters = off; off = align256(off + 4ull * B);
    h.decode_ws = off;
    h.total = align256(off + lbp_workspace_size(c, prm, B));
    h.llr = h.total;
    h.total_llr = h.llr + align256(4ull * c->n * B);
    return h;
}

}  // namespace

extern "C" size_t lbp_host_workspace_size(const lbp_code *code, const lbp_params *params, int64_t num_shots) {
    if (check_common(code, params, num_shots)) return 0;
    if (lbp_workspace_size(code, params, num_shots) == 0) return 0;
    return host_stage(code, params, num_shots).total;
}

extern "C" int lbp_decode_host(const lbp_code *code, const lbp_params *params, int64_t num_shots,
                               const uint64_t *syndromes, uint64_t *err_out, uint8_t *converged,
                               uint8_t *osd_out, int32_t *iters_out, float *llr_out,
                               void *workspace, size_t workspace_bytes, void *stream) {
    int rc = check_common(code, params, num_shots);
    if (rc) return rc;
    if (num_shots == 0) return LBP_OK;
    if (!syndromes || !err_out || !converged || !iters_out || !workspace) return LBP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != code->device) return LBP_EINVAL;
    const HostStage h = host_stage(code, params, num_shots);
    if (workspace_bytes < (llr_out ? h.total_llr : h.total)) return LBP_ENOMEM;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return LBP_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *base = static_cast<uint8_t *>(workspace);
    const int64_t B = num_shots;
    const size_t wm = (code->m + 63) / 64, wn = (code->n + 63) / 64;
    uint64_t *d_syn = reinterpret_cast<uint64_t *>(base + h.syn);
    uint64_t *d_err = reinterpret_cast<uint64_t *>(base + h.err);
    uint8_t *d_conv = base + h.conv;
    uint8_t *d_osd = base + h.osd;
    int32_t *d_iters = reinterpret_cast<int32_t *>(base + h.iters);
    float *d_llr = llr_out ? reinterpret_cast<float *>(base + h.llr) : nullptr;
    // Outputs of shots [s0, s0 + nb) to the host, on stream q.
    auto d2h = [&](int64_t s0, int64_t nb, cudaStream_t q) {
        bool ok = cudaMemcpyAsync(err_out + s0 * wn, d_err + s0 * wn, 8ull * wn * nb, cudaMemcpyDeviceToHost,
                                  q) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(converged + s0, d_conv + s0, static_cast<size_t>(nb), cudaMemcpyDeviceToHost,
                                   q) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(iters_out + s0, d_iters + s0, 4ull * nb, cudaMemcpyDeviceToHost, q) == cudaSuccess;
        if (osd_out)
            ok = ok && cudaMemcpyAsync(osd_out + s0, d_osd + s0, static_cast<size_t>(nb), cudaMemcpyDeviceToHost,
                                       q) == cudaSuccess;
        if (llr_out)
            ok = ok && cudaMemcpyAsync(llr_out + s0 * code->n, d_llr + s0 * code->n, 4ull * code->n * nb,
                                       cudaMemcpyDeviceToHost, q) == cudaSuccess;
        return ok;
    };
    const int K = B >= 4 * kHostChunkShots ? 4 : (B >= 2 * kHostChunkShots ? 2 : 1);
    CopyStreams cs;
    if (K == 1 || !copy_streams(dev, &cs)) {
        if (cudaMemcpyAsync(d_syn, syndromes, 8ull * wm * B, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            return LBP_ECUDA;
        }
        rc = decode_device(code, params, B, d_syn, d_err, d_conv, d_osd, d_iters, d_llr,
                           base + h.decode_ws, h.total - h.decode_ws, s);
        if (rc) return rc;
        if (!d2h(0, B, s)) { cudaGetLastError(); return LBP_ECUDA; }
        return LBP_OK;
    }
    // Pipeline over K consecutive chunks: every host-to-device copy is queued
    // on the input copy stream at once, chunk i decodes on the caller's stream
    // after its input arrived (shot_offset advanced, so each shot draws as in
    // one call), and its outputs leave on the output copy stream while the
    // next chunk decodes.  Events order the copy streams after the caller's
    // earlier work, and the caller's stream after the last copy.
    cudaEvent_t ev[2 * 4 + 2] = {};
    auto release = [&]() {
        for (cudaEvent_t &e : ev)
            if (e) cudaEventDestroy(e);
    };
    for (cudaEvent_t &e : ev) {
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            release();
            return LBP_ECUDA;
        }
    }
    cudaEvent_t ev_start = ev[0], ev_end = ev[1], *ev_in = ev + 2, *ev_dec = ev + 2 + K;
    bool ok = cudaEventRecord(ev_start, s) == cudaSuccess;
    ok = ok && cudaStreamWaitEvent(cs.in, ev_start, 0) == cudaSuccess;
    ok = ok && cudaStreamWaitEvent(cs.out, ev_start, 0) == cudaSuccess;
    const int64_t chunk = (B + K - 1) / K;
    for (int i = 0; ok && i < K; ++i) {
        const int64_t s0 = i * chunk, nb = std::min<int64_t>(chunk, B - s0);
        ok = cudaMemcpyAsync(d_syn + s0 * wm, syndromes + s0 * wm, 8ull * wm * nb, cudaMemcpyHostToDevice,
                             cs.in) == cudaSuccess;
        ok = ok && cudaEventRecord(ev_in[i], cs.in) == cudaSuccess;
    }
    for (int i = 0; ok && i < K; ++i) {
        const int64_t s0 = i * chunk, nb = std::min<int64_t>(chunk, B - s0);
        lbp_params p = *params;
        p.shot_offset += static_cast<uint64_t>(s0);
        ok = cudaStreamWaitEvent(s, ev_in[i], 0) == cudaSuccess;
        if (ok) {
            rc = decode_device(code, &p, nb, d_syn + s0 * wm, d_err + s0 * wn, d_conv + s0, d_osd + s0,
                               d_iters + s0, d_llr ? d_llr + s0 * code->n : nullptr, base + h.decode_ws,
                               h.total - h.decode_ws, s);
            if (rc) break;
        }
        ok = ok && cudaEventRecord(ev_dec[i], s) == cudaSuccess;
        ok = ok && cudaStreamWaitEvent(cs.out, ev_dec[i], 0) == cudaSuccess;
        ok = ok && d2h(s0, nb, cs.out);
    }
    ok = ok && cudaEventRecord(ev_end, cs.out) == cudaSuccess;
    ok = ok && cudaStreamWaitEvent(s, ev_end, 0) == cudaSuccess;
    if (rc || !ok) {
        // The pipeline stopped early: order the caller's stream after every
        // copy already queued on the copy streams, so that the caller may
        // reuse its buffers and the workspace once its stream has drained.
        for (cudaStream_t q : {cs.in, cs.out})
            if (cudaEventRecord(ev_start, q) == cudaSuccess) cudaStreamWaitEvent(s, ev_start, 0);
    }
    release();
    if (rc) return rc;
    if (!ok) { cudaGetLastError(); return LBP_ECUDA; }
    return LBP_OK;
}

// ---- Merged launch: one BP launch over the shots of several requests ------

namespace {

constexpr int kMaxBatchItems = 64;

struct BatchPlan {
    int n = 0, msg = 0, DC = 0, DV = 0, S = 0, G = 0, grid = 0;
    int64_t total = 0;
    size_t smem = 0;
    uint32_t state_bytes = 0;
    size_t off_items = 0, total_ws = 0;
    size_t item_off[kMaxBatchItems];
    WsLayout w[kMaxBatchItems];
    OsdPlan op[kMaxBatchItems];
    OsdWarpPlan wp[kMaxBatchItems];
    uint32_t off_lam[kMaxBatchItems], off_s[kMaxBatchItems], off_shat[kMaxBatchItems];
};

// Plan a merged launch: every item valid and of one message type, the
// min-sum rule, a 16-bit index image and the same degree bounds; the
// groups' states sized for the largest code; workspace = the launch's
// counters, the device copy of the item array, then each item's own
// lbp_decode workspace (its OSD counters, queue and pools).
int plan_batch(const lbp_batch_item *items, int n, BatchPlan *P, bool size_only = false) {
    if (!items || n < 1 || n > kMaxBatchItems) return LBP_EINVAL;
    P->n = n;
    P->msg = items[0].params.msg;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return LBP_ECUDA; }
    uint32_t maxst = 16;
    int maxpairs = 1;
    for (int i = 0; i < n; ++i) {
        const lbp_batch_item &it = items[i];
        const int rc = check_common(it.code, &it.params, it.num_shots);
        if (rc) return rc;
        if (!size_only && it.num_shots > 0 && (!it.syndromes || !it.err_out || !it.converged || !it.iters_out))
            return LBP_EINVAL;
        if (it.code->device != dev) return LBP_EINVAL;
        const lbp_code *c = it.code;
        if (it.params.msg != P->msg || it.params.rule != LBP_RULE_MIN_SUM) return LBP_ENOSYS;
        if (it.params.lottery_policy == LBP_LOTTERY_PROPOSED_CURRENT) return LBP_ENOSYS;
        if (!c->d_ell || c->ell.idx_bytes != 2) return LBP_ENOSYS;
        if (i == 0) { P->DC = c->ell.DC; P->DV = c->ell.DV; }
        if (c->ell.DC != P->DC || c->ell.DV != P->DV) return LBP_ENOSYS;
        const int W32 = (c->m + 31) / 32;
        const int R = c->tab_R > 0 ? c->tab_R : c->ell.Mp + 2;   // the stride of the image's offsets
        uint32_t o = align16u(static_cast<uint32_t>(msg_bytes(P->msg)) * P->DC * R);
        P->off_lam[i] = o;  o = align16u(o + 4u * (c->ell.Np + 2));
        P->off_s[i] = o;    o = align16u(o + 4u * W32);
        P->off_shat[i] = o; o = align16u(o + 12u * W32);
        if (o > maxst) maxst = o;
        maxpairs = std::max(maxpairs, std::max(c->ell.Mp, c->ell.Np) / 2);
        P->total += it.num_shots;
    }
    if (P->total > (1ll << 31)) return LBP_EINVAL;
    const lbp_code *c0 = items[0].code;
    P->state_bytes = maxst;
    // Groups per CTA: as many states (plus their 16-byte shot slots) as fit,
    // at most 15 named barriers; threads per group: about one per six pairs
    // of the largest code's checks or columns (64, 128 or 192), narrowed so
    // the CTA keeps at most 1024 threads.
    const size_t budget = static_cast<size_t>(c0->smem_optin);
    int S = static_cast<int>(budget / (static_cast<size_t>(maxst) + 16));
    if (S < 1) return LBP_ENOSYS;
    if (S > 15) S = 15;
    int G = maxpairs > 6 * 128 ? 192 : (maxpairs > 6 * 64 ? 128 : 64);
    while (G > 64 && S * G > 1024) G = G == 192 ? 128 : 64;
    if (S * G > 1024) S = 1024 / G;
    P->S = S;
    P->G = G;
    P->smem = static_cast<size_t>(S) * (16 + maxst);
    const int64_t need = (P->total + S - 1) / S;
    P->grid = static_cast<int>(need < c0->sm_count ? need : c0->sm_count);
    if (P->grid < 1) P->grid = 1;
    size_t off = align256(256);
    P->off_items = off;
    off = align256(off + sizeof(BpEllArgs) * n);
    for (int i = 0; i < n; ++i) {
        const lbp_batch_item &it = items[i];
        if (it.params.osd) {
            int rc = plan_osd(it.code, it.num_shots, &P->op[i]);
            if (rc) return rc;
            plan_osd_warp(it.code, it.num_shots, &P->wp[i]);
        }
        P->w[i] = layout(it.code, &it.params, it.num_shots, it.params.osd ? &P->op[i] : nullptr,
                         it.params.osd ? &P->wp[i] : nullptr, nullptr);
        P->item_off[i] = off;
        off = align256(off + P->w[i].total);
    }
    P->total_ws = off;
    return LBP_OK;
}

}  // namespace

namespace lbp {

size_t batch_workspace_size(const lbp_batch_item *items, int n_items) {
    BatchPlan P;
    if (plan_batch(items, n_items, &P, true)) return 0;
    return P.total_ws;
}

}  // namespace lbp

extern "C" size_t lbp_batch_workspace_size(const lbp_batch_item *items, int32_t n_items) {
    return lbp::batch_workspace_size(items, n_items);
}

extern "C" int lbp_decode_batch(const lbp_batch_item *items, int32_t n_items, void *workspace,
                                size_t workspace_bytes, void *stream) {
    BatchPlan P;
    int rc = plan_batch(items, n_items, &P);
    if (rc) return rc;
    if (!workspace || workspace_bytes < P.total_ws) return LBP_ENOMEM;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return LBP_EINVAL;
    if (P.total == 0) return LBP_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t *base = static_cast<uint8_t *>(workspace);
    unsigned int *counters = reinterpret_cast<unsigned int *>(base);
    if (cudaMemsetAsync(counters, 0, 256, st) != cudaSuccess) { cudaGetLastError(); return LBP_ECUDA; }
    std::vector<BpEllArgs> h(static_cast<size_t>(n_items));
    int64_t first = 0;
    for (int i = 0; i < n_items; ++i) {
        const lbp_batch_item &it = items[i];
        const lbp_code *c = it.code;
        uint8_t *ib = base + P.item_off[i];
        unsigned int *ictr = reinterpret_cast<unsigned int *>(ib + P.w[i].counters);
        if (cudaMemsetAsync(ictr, 0, 256, st) != cudaSuccess) { cudaGetLastError(); return LBP_ECUDA; }
        BpEllArgs &e = h[i];
        std::memset(&e, 0, sizeof(e));
        e.image = c->d_ell;
        e.img = c->ell;
        e.m = c->m; e.n = c->n;
        e.max_iter = it.params.max_iter; e.scale_mode = it.params.scale_mode; e.scale_const = it.params.scale_const;
        e.lottery = it.params.lottery; e.lottery_skip = it.params.lottery_skip; e.osd = it.params.osd;
        e.policy = it.params.lottery_policy; e.rule = it.params.rule;
        e.seed = it.params.seed; e.shot_offset = it.params.shot_offset;
        e.num_shots = it.num_shots;
        e.syn = it.syndromes; e.err = it.err_out; e.conv = it.converged; e.osd_out = it.osd_out;
        e.iters = it.iters_out; e.llr = nullptr;
        e.counters = ictr;
        e.osd_list = it.params.osd ? reinterpret_cast<uint32_t *>(ib + P.w[i].osd_list) : nullptr;
        e.osd_llr = it.params.osd ? reinterpret_cast<float *>(ib + P.w[i].osd_llr) : nullptr;
        e.state_bytes = P.state_bytes;
        e.off_beta = 0; e.off_lam = P.off_lam[i]; e.off_s = P.off_s[i]; e.off_shat = P.off_shat[i];
        const int R = c->tab_R > 0 ? c->tab_R : c->ell.Mp + 2;
        e.tab_R = c->tab_R;
        e.magic = static_cast<uint32_t>((1ull << 32) / static_cast<uint64_t>(R) + 1);
        e.first = first;
        first += it.num_shots;
    }
    BpEllArgs *d_items = reinterpret_cast<BpEllArgs *>(base + P.off_items);
    // Pageable source: the call returns once the array is staged for the copy.
    if (cudaMemcpyAsync(d_items, h.data(), sizeof(BpEllArgs) * h.size(), cudaMemcpyHostToDevice, st) !=
        cudaSuccess) {
        cudaGetLastError();
        return LBP_ECUDA;
    }
    BpEllArgs a = h[0];                       // item 0's image and sizes, for the kernel's prologue
    a.counters = counters;
    a.num_shots = P.total;
    a.state_bytes = P.state_bytes;
    a.items = d_items;
    a.n_items = n_items;
    const LaunchShape shp{P.grid, P.S, P.G, P.smem, false, true, false, false, false, false, true};
    void *tk = timing_begin(st);
    switch (P.msg) {
        case LBP_MSG_F32: rc = launch_bp_ell_f32(shp, a, P.DC, P.DV, st); break;
        case LBP_MSG_F16: rc = launch_bp_ell_f16(shp, a, P.DC, P.DV, st); break;
        default: rc = launch_bp_ell_i8(shp, a, P.DC, P.DV, st); break;
    }
    timing_end(tk, st, kTimeBp);
    if (rc) return rc;
    rc = check_launch();
    if (rc) return rc;
    for (int i = 0; i < n_items && rc == LBP_OK; ++i) {
        const lbp_batch_item &it = items[i];
        if (!it.params.osd || it.num_shots == 0) continue;
        uint8_t *ib = base + P.item_off[i];
        rc = launch_osd(it.code, it.num_shots, it.syndromes, it.err_out, it.osd_out,
                        reinterpret_cast<unsigned int *>(ib + P.w[i].counters), ib, P.w[i], P.op[i], P.wp[i],
                        h[i].osd_list, h[i].osd_llr, st, false);
    }
    return rc;
}

extern "C" int lbp_code_tuned(const lbp_code *code, int32_t msg, int32_t rule, int32_t *groups, int32_t *G,
                              int32_t *graph) {
    if (!code || msg < 0 || msg > 2 || (rule != LBP_RULE_MIN_SUM && rule != LBP_RULE_SUM_PRODUCT)) return LBP_EINVAL;
    const int mi = tuned_slot(msg, rule);
    if (groups) *groups = code->tuned_groups[mi];
    if (G) *G = code->tuned_G[mi];
    if (graph) *graph = code->tuned_graph[mi];
    return LBP_OK;
}

extern "C" int lbp_tune(lbp_code *code, const lbp_params *params, int64_t num_shots,
                        const uint64_t *syndromes, uint64_t *err_out, uint8_t *converged,
                        uint8_t *osd_out, int32_t *iters_out, void *workspace, size_t workspace_bytes,
                        void *stream) {
    int rc = check_common(code, params, num_shots);
    if (rc) return rc;
    if (num_shots == 0) return LBP_OK;
    if (!syndromes || !err_out || !converged || !iters_out) return LBP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != code->device) return LBP_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int mi = tuned_slot(params->msg, params->rule);
    code->tuned_G[mi] = 0;
    code->tuned_groups[mi] = 0;
    code->tuned_graph[mi] = 0;
    const int Gs[] = {32, 64, 96, 128, 192, 256, 512, 768, 1024};
    float best = -1.0f;
    int best_S = 0, best_G = 0, best_graph = 0;
    // Candidates: every thread count, with the index image and, for a
    // recognised surface code, with the implicit graph.
    std::vector<std::pair<int, int>> seen;           // (S, G) already timed for this graph form
    for (int graph = 1; graph <= 3; ++graph) {
        if (graph == 2 && !code->surface) continue;
        if (graph == 3 && !code->round) continue;
        seen.clear();
        for (int cand = 0; cand < 2 * static_cast<int>(sizeof(Gs) / sizeof(Gs[0])); ++cand) {
            // Each width with as many groups as fit, then with one group per CTA.
            const int G = Gs[cand % (sizeof(Gs) / sizeof(Gs[0]))];
            const int S_req = cand < static_cast<int>(sizeof(Gs) / sizeof(Gs[0])) ? 1024 : 1;
            BpPlan probe;
            if (plan_bp(code, params->msg, params->rule, num_shots, &probe, S_req, G, graph) != LBP_OK) continue;
            if (probe.G != G) continue;                    // shape not available for this code
            const int S = probe.groups;
            if (std::find(seen.begin(), seen.end(), std::make_pair(S, G)) != seen.end()) continue;
            seen.emplace_back(S, G);
            float ms = 0.0f, warm = 0.0f;
            rc = lbp::decode_device_shaped(code, params, num_shots, syndromes, err_out, converged, osd_out,
                                           iters_out, nullptr, workspace, workspace_bytes, s, S, G, &warm,
                                           graph);
            if (rc == LBP_ENOMEM || rc == LBP_ENOSYS) continue;   // candidate does not fit: skip it
            if (rc) return rc;
            rc = lbp::decode_device_shaped(code, params, num_shots, syndromes, err_out, converged, osd_out,
                                           iters_out, nullptr, workspace, workspace_bytes, s, S, G, &ms, graph);
            if (rc) return rc;
            // Two timed runs, the faster kept: close candidates (a few %
            // apart) are otherwise picked by timing noise.
            float ms2 = 0.0f;
            rc = lbp::decode_device_shaped(code, params, num_shots, syndromes, err_out, converged, osd_out,
                                           iters_out, nullptr, workspace, workspace_bytes, s, S, G, &ms2, graph);
            if (rc) return rc;
            if (ms2 > 0.0f && (ms <= 0.0f || ms2 < ms)) ms = ms2;
            if (ms > 0.0f && (best < 0.0f || ms < best)) { best = ms; best_S = S; best_G = G; best_graph = graph; }
        }
    }
    if (best_G > 0) {
        code->tuned_G[mi] = best_G;
        code->tuned_groups[mi] = best_S;
        code->tuned_graph[mi] = best_graph;
    } else {
        // No candidate ran: decode once with the default shape so the outputs
        // are lbp_decode's (or report why it cannot run).
        rc = lbp::decode_device(code, params, num_shots, syndromes, err_out, converged, osd_out,
                                iters_out, nullptr, workspace, workspace_bytes, s);
        if (rc) return rc;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); return LBP_ECUDA; }
    return LBP_OK;
}
