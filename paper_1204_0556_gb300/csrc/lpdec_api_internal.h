// Host-side internals shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "lpdec.h"
#include "lpdec_internal.h"

namespace lpdec {

// Tile shape: `groups` frames decoded concurrently per CTA, each by a group of
// `group_threads` threads (one check per thread per pass).
struct Tile {
    int groups = 1;
    int group_threads = 32;
    int ring = 0;        // STREAMED only: state slots of the producer-warp ring (0: plain kernel)
    bool valid = false;  // set when chosen by the autotuner or by hand
};

struct SliceLayout {
    size_t off_x = 0, off_red = 0, bytes = 0;
};

int set_error(int code, const char *fmt, ...);
// Stream-ordered allocation from the library's per-device memory pool (freed
// with cudaFreeAsync; the pool keeps the memory for later calls).
cudaError_t lib_alloc(void **ptr, size_t bytes, cudaStream_t stream);
int cuda_error(cudaError_t e, const char *what);
int validate_params(const lpdec_params *p);
IterCfg make_cfg(const lpdec_code *c, const lpdec_params *p);
CodeView make_view(const lpdec_code *c);
SliceLayout slice_layout(const lpdec_code *c, int dtype, int group_threads);
// max_threads > 0 caps the CTA size (kernels built for smaller CTAs).
Tile default_tile(const lpdec_code *c, int dtype, int max_threads = 0);
// The tile a decode with these parameters uses: the tuned tile of its schedule
// (STREAMED has its own), else the RESIDENT one, else the default.
Tile chosen_tile(const lpdec_code *c, const lpdec_params *p);
int device_smem_optin(int device);
int device_sm_count(int device);
// Fills lc and (plain kernel) the slice layout or (ring kernel) the layout of
// a group's scratch; a ring tile needs STREAMED state (k_state != null).
int plan_launch(const lpdec_code *c, int dtype, const Tile &tile, int n_frames, cudaStream_t stream,
                LaunchCfg *lc, SliceLayout *layout);
// Copies the tile, layout and launch geometry into the kernel arguments.
void apply_plan(DecodeArgs &a, const Tile &tile, const LaunchCfg &lc, const SliceLayout &L);
// Least shared memory a ring tile needs (indices not staged, slots without the
// LLR row); 0 if it is not a valid ring tile.
size_t ring_smem_bytes(const lpdec_code *c, int dtype, const Tile &tile);
int resolve_schedule(const lpdec_code *c, const lpdec_params *p, const Tile &tile);
size_t workspace_bytes(const lpdec_code *c, int n_frames, int schedule, int dtype, int max_iter, int ipl);
int launch_once(const lpdec_code *c, int dtype, const Tile &tile, DecodeArgs &a, cudaStream_t stream);
int enqueue_decode(const lpdec_code *c, int n_frames, const float *llr, const lpdec_params *p, float *x_out,
                   uint8_t *bits_out, int32_t *iters_out, uint8_t *cert_out, cudaStream_t stream, void *work,
                   int schedule, const Tile &tile, int *launches_out);

}  // namespace lpdec

struct lpdec_code {
    int n = 0, m = 0, E = 0, Ep = 0;
    int max_dc = 0, k_rank = 0, cls = 0, device = 0;
    int reg_dv = 0;             // variable degree if the code runs the regular-code kernel, else 0
    int reg_dc = 0;             // its common check degree, or 0 when check degrees differ (wide classes)
    void *dev_block = nullptr;  // one allocation holding the four index arrays
    int32_t *row_ptr = nullptr, *col_idx = nullptr, *col_ptr = nullptr, *csc_edge = nullptr;
    int32_t *check_order = nullptr;  // wide classes with differing check degrees (see CodeView), else null
    // Regular codes: 16-bit index block (CodeView::col16 / csc16), else null.
    void *dev_idx16 = nullptr;
    int idx16_bytes = 0, col16_elems = 0;
    lpdec::Tile tuned[4];           // per state dtype, from lpdec_autotune (RESIDENT) or lpdec_set_tile
    lpdec::Tile tuned_streamed[4];  // per state dtype, from lpdec_autotune (STREAMED) or lpdec_set_tile
    lpdec::Tile dual_tile;  // tile of the dual subgradient decoder, from lpdec_dual_set_tile
};
