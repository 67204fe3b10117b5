// Internal definitions shared by the host and device parts of liblbp.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "lbp.h"

namespace lbp {

constexpr int kMaxRowDeg = 32;      // a check's neighbours fit one warp / one 32-bit mask
constexpr int kMaxIter = (1 << 24) - 1;

// Byte offsets of the compact graph image that each decoding CTA copies into
// shared memory.  All index arrays are uint16 (the image exists only when
// m, n and nnz are all below 65536); mu is binary32.
struct GraphImage {
    uint32_t bytes;          // total, a multiple of 16
    uint32_t off_row_ptr;    // u16[m+1]   CSR row starts
    uint32_t off_col_idx;    // u16[nnz]   CSR column of each edge
    uint32_t off_col_ptr;    // u16[n+1]   CSC column starts
    uint32_t off_csc_edge;   // u16[nnz]   CSR edge id of each CSC entry (rows ascending)
    uint32_t off_csc_row;    // u16[nnz]   check of each CSC entry
    uint32_t off_mu;         // f32[n]     prior LLR
};

// ELL image for bounded-degree codes (bp_ell_kernel), with Mp, Np = m, n
// rounded up to even and R = Mp + 2: check side cidx[DC][Mp] (column ids,
// padding n) and column side vent[DV][Np] (message offset slot * R + check,
// padding Mp), both slot-major uint16, then mu[Np + 2] with mu[n] = +inf.
// Exists when every check has <= 8 ones, every column <= 4, DC * R < 65536 and
// n < 65535.
struct EllImage {
    uint32_t bytes;
    uint32_t off_cidx, off_vent, off_mu;
    int32_t DC, DV;
    int32_t Mp, Np;          // m and n rounded up to even (paired accesses)
    int32_t idx_bytes;       // 2 (uint16 indices) or 4 (uint32, image read from global memory)
    // Slot-aligned layout (space-time matrices whose image and FP32 state do
    // not fit shared memory together): every check's round columns in slots
    // 0 .. DC-3, its measurement columns of blocks t-1 and t in slots DC-2
    // and DC-1; meas0 = the first measurement column (0: not aligned).
    int32_t meas0;
};

// Space-time matrix of the unrotated surface code (Eq. 1 with one check type
// per round), recognised by lbp_load_code: T rounds of m_r = d(d-1) checks
// over n_r = d^2 + (d-1)^2 data columns, then nb measurement blocks of m_r
// columns (nb = T - 1 with an open time boundary, T when cyclic).  Table III
// gives each check's columns by closed formulas; the BP kernel evaluates them
// (and their inverses for the column side) instead of loading an index image.
struct SurfaceDesc {
    int32_t d, T, nb;
    int32_t type;            // 0: X checks (H_X rows), 1: Z checks (H_Z rows)
    int32_t cyclic;
    uint32_t nr, mr, d2;     // n_r, m_r, d^2
    uint32_t mg_d, mg_d1, mg_nr, mg_mr;   // floor(2^32 / x) + 1 for exact x / divisor
    int32_t mu_uniform;      // 1: mu is one value on data columns and one on measurement columns
    float mu_data, mu_meas;
};

// Space-time matrix of Eq. 1 for any per-round check matrix H_r (m_r x n_r):
// rows t m_r + j (t < T) hold H_r's row j shifted by t n_r plus the
// measurement columns T n_r + b m_r + j of blocks b = t - 1 and b = t that
// exist (nb = T - 1 blocks with an open time boundary, T when cyclic).
// Recognised by lbp_load_code for every H of that form; the BP kernel then
// stores one round's index table instead of the whole graph.
// Round image: rcidx[DC - 2][m_r] (uint16) the round columns of each round
// check in ascending order (n_r when absent), then rvent[DV][n_r] (uint32)
// slot * R + j of each round column's round checks ascending (~0 when
// absent).  A check's slots are its round columns (0 .. DC - 3), then the
// measurement blocks t - 1 (slot DC - 2) and t (slot DC - 1).
struct RoundDesc {
    int32_t T, nb, cyclic;
    uint32_t mr, nr;
    uint32_t mg_mr, mg_nr;   // floor(2^32 / x) + 1 for exact x / divisor
    uint32_t bytes, off_rcidx, off_rvent;
    int32_t mu_uniform;
    float mu_data, mu_meas;
};

}  // namespace lbp

struct lbp_code;

namespace lbp {

// Per-shot state of the ELL kernel: messages [DC][R], posteriors [Np + 2],
// syndrome words, three s_hat buffers, and 16 bytes of group scratch, each
// part 16-byte aligned.
inline uint32_t ell_state_bytes(int msg_bytes, int DC, int R, int Np, int m) {
    auto a16 = [](uint32_t x) { return (x + 15u) & ~15u; };
    const uint32_t W32 = static_cast<uint32_t>((m + 31) / 32);
    uint32_t off = a16(static_cast<uint32_t>(msg_bytes) * DC * R);
    off = a16(off + 4u * (Np + 2));
    off = a16(off + 4u * W32);
    off = a16(off + 12u * W32);
    return a16(off + 16u);
}

// The decode path behind lbp_decode: plan, workspace layout and launches of
// K_bp and the OSD kernels on `stream`, using `ws_bytes` bytes at `ws`
// (device, 256-byte aligned) as scratch.  Parameters are already validated.
// alone: nothing else runs on the device meanwhile, so a batch of at most one
// shot per SM may take the latency layouts (a CTA per shot with up to 1024
// BP threads; OSD with one warp and the whole shared memory per CTA), which
// would crowd out concurrent work.
int decode_device(const lbp_code *c, const lbp_params *prm, int64_t B, const uint64_t *syn,
                  uint64_t *err, uint8_t *conv, uint8_t *osd_out, int32_t *iters, float *llr,
                  void *ws, size_t ws_bytes, cudaStream_t stream, bool alone = true);

// Same, with an explicit BP launch shape (groups per CTA, threads per group;
// 0, 0 = the code's tuned or default shape) and graph form (1 index image,
// 2 implicit surface-code graph, 0 = tuned or default); when bp_ms is
// non-null the BP kernel is timed with an event pair on `stream` (the call
// then waits).
int decode_device_shaped(const lbp_code *c, const lbp_params *prm, int64_t B, const uint64_t *syn,
                         uint64_t *err, uint8_t *conv, uint8_t *osd_out, int32_t *iters, float *llr,
                         void *ws, size_t ws_bytes, cudaStream_t stream, int groups, int G,
                         float *bp_ms, int graph = 0, bool alone = true);

// Device workspace bytes of a merged launch of these items (0 if they cannot
// share one); the buffer pointers are not looked at.
size_t batch_workspace_size(const lbp_batch_item *items, int n_items);

}  // namespace lbp

struct lbp_code {
    int device;
    int sm_count;
    int smem_optin;          // max dynamic shared memory per block
    int32_t m, n, nnz;
    int32_t max_row_deg, max_col_deg;
    // Compact image (device), NULL when the sizes do not fit 16-bit indices.
    uint8_t *d_image;
    lbp::GraphImage img;
    // ELL image (device), NULL when the code's degrees or sizes exceed it.
    uint8_t *d_ell;
    lbp::EllImage ell;
    // Bank-aware layout of the index-image form, for codes whose image and
    // FP32 state always fit in shared memory (0 otherwise): message rows of
    // tab_R words (a multiple of 32) and, at image offset tab_off_ptab, the
    // table of check pairs in the order the kernel's lanes take them.
    int32_t tab_R;
    uint32_t tab_off_ptab;
    // 32-bit device copies, used by OSD.
    int32_t *d_row_ptr, *d_col_idx;
    float *d_mu;
    // Implicit graph (Table III) when H is a recognised surface-code
    // space-time matrix; d_mu_pad is mu[Np + 2] with +inf past n.
    int surface;
    lbp::SurfaceDesc surf;
    float *d_mu_pad;
    // Round-periodic graph (Eq. 1 with any round matrix) and its round image.
    int round;
    lbp::RoundDesc rnd;
    uint8_t *d_round;
    // BP launch shape chosen by lbp_tune per message type (0 = not tuned):
    // groups per CTA and threads per group.
    int tuned_groups[6], tuned_G[6];   // per (rule, message type), lbp_tune
    int tuned_graph[6];                // graph form chosen by lbp_tune (0 none, 1 image, 2 implicit)
    // Experiment switches, read from the environment once, by lbp_load_code,
    // so that decodes of a loaded code never depend on the environment at
    // call time: LBP_GRAPH (0 unset, 1 table, 2 implicit, 3 round),
    // LBP_BP_SHAPE "S,G" (0, 0 unset), LBP_OSD_POOL_ROWS (0 unset) and
    // LBP_OSD_LAT (0: latency layout off), LBP_OSD_DENSE (0: dense OSD off),
    // LBP_BANK_LAYOUT (0: bank-aware index image off).
    int env_graph, env_S, env_G, env_pool_rows, env_osd_lat, env_osd_dense, env_bank_layout;
    // Dense OSD (K_osd_dense) for codes with m <= 160 and n + 1 <= 320 and a
    // 16-bit image: rows per lane, 64-bit words per augmented row, rank(H)
    // over GF(2); osd_dense = 0 when the code takes the event-driven kernels.
    int osd_dense, osd_RL, osd_WN;
    int32_t osd_rank;
};
