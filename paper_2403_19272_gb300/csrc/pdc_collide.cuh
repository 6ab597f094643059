// Collision data structures and kernel entry points.
#pragma once
#include <algorithm>

#include "pdc_internal.cuh"
#include "pdc_prof.cuh"

namespace pdc {

enum OverflowBits { OVF_HASH = 1, OVF_VT = 2, OVF_EE = 4, OVF_ACTIVE = 8, OVF_CELLS = 16, OVF_SLOTS = 32 };

// Cells are boxes whose side along each axis follows the mean swept-box
// extent of the triangles along that axis (boxes stretched by the motion
// get cells stretched the same way).
struct GridParams {
    double ext_sum[3];  // per axis: sum over triangles of the swept-box extent
    float cell[3], inv_cell[3];
};

// Collision settings shared by the pair kernels.
struct CollParams {
    float dhat;       // activity gap / contact target gap
    double eta;       // exact-CCD contact distance
    float k_ndb;      // initial weight k of Eq. (exp)
    float K_ndb;      // growth base K
    int a_max;        // cap of the life-span counter
    int samples_vt;   // 0, 1, 3
    int samples_ee;   // 0, 1, 4
    int adaptive;     // 1: sample lattice per pair from the bound of Eq. (sample_bound)
    int max_axis;     // cap on that lattice's samples per parameter axis
    double alpha;     // line-search factor alpha of the bound
};

// An active collision constraint: 4 collision-vertex ids, the gap-vector
// coefficients c (p2 - p1 = sum_j c_j x_j at the t = 0 closest points), the
// unit start direction n0 and the NDB weight w.
struct ActivePair {
    int4 ids;
    float4 c;
    float4 n0w;
};

// Pair state byte: bit 7 = active, bits 0..6 = life-span counter a.
constexpr unsigned char ST_ACTIVE = 0x80;

// Bookkeeping of the partial-CCD filter (device).  A pair can pass the
// activity test only if its start distance d0 is within d_hat plus the
// largest relative displacement of its vertices since x^- ("near").  A full
// pass over the list measures each pair's margin to that bound; pairs whose
// margin exceeds the watch gap tau stay non-near until some vertex has moved
// by more than tau/2 since that pass, so until then only the watch list
// (margin < tau) is scanned.
struct PccdState {
    unsigned int amax_bits;  // max_v |disp_v - disp0_v| since the last full pass (float bits)
    int n_near;              // near pairs found by this pass
    int n_watch_new;         // watch list being written by this (full) pass
    int pass_full;           // this pass scans every pair
    int force_full;          // the lists changed: the next pass must be full
    int watch_ok;            // the current watch list is complete
    int n_watch;             // current watch list length
    int cur;                 // which watch buffer is current
};

// Broad phase (Sec. 4 candidate pairs, culled by a uniform grid): one hash
// table of grid cells holding every collision vertex, edge and triangle over
// the cells its swept box covers, the box's upper side raised by d_hat; the
// VT and EE pairs of each cell are tested from shared memory.
struct BroadPhase {
    int nt = 0, ne = 0, nv = 0;
    int T = 0;  // buckets of the cell table (power of two)
    long long cap_ent = 0, cap_vt = 0, cap_ee = 0;
    float cell_scale = 1.f;  // grown x4 when a primitive covers too many cells
    float cell_grid = 1.f;   // tuned factor of the cell side (1, 1.5 or 2)
    DevBuf<int> bcnt, bstart, bfill;
    DevBuf<unsigned long long> ekey;  // cell key of each table entry
    DevBuf<unsigned int> epay;        // primitive | kind << 27 | lowest-cell flags << 29
    DevBuf<unsigned long long> equ;   // the entry's box quantized within its cell (two words)
    DevBuf<int> work;                 // bucket counter of the cell-pair kernel
    DevBuf<float4> tlo, thi, elo, ehi;
    DevBuf<int> cnt_v, cnt_e, scratch;
    // per list buffer: offset of each primary's segment in that list (the
    // prefix sum of the counts), valid when the list came from a hash pass
    // (off_ok), so that the next full CCD finds a pair's old state in its
    // primary's segment instead of by binary search over the whole list
    DevBuf<int> off_v[2], off_e[2];
    bool off_ok[2] = {false, false};
    DevBuf<int> slots_vt, slots_ee;  // per-primary candidate rows (sorted when compacted)
    int w_vt = 16, w_ee = 32;        // row widths (doubled on OVF_SLOTS)
    DevBuf<GridParams> gp;
    DevBuf<long long> totals;
    // double-buffered candidate lists and NDB pair states
    DevBuf<int2> vt[2], ee[2];
    DevBuf<unsigned char> st_vt[2], st_ee[2];
    DevBuf<float> d0_vt[2], d0_ee[2];  // per pair: closest distance on x^- (partial-CCD prefilter)
    DevBuf<long long> cnt_vt_d[2], cnt_ee_d[2];
    int cur = 0;
    unsigned gen = 0;          // counts reallocations of the buffers below (captured graphs go stale)
    // launch shapes (autotuned at the first step when asked): blocks of the
    // pair kernels and warps per block of the cell-pair kernel; with tune_*
    // set, the next launch times every candidate on its own data and keeps
    // the fastest
    int pair_blocks = 152 * 8;
    int cell_warps = 8;
    bool tune_pairs = false, tune_cells = false;
    int tune_wait = 0;  // passes since tune_cells was set
    float pair_ms[4] = {0, 0, 0, 0}, cell_ms[3] = {0, 0, 0}, grid_ms[3] = {0, 0, 0};
    Profiler *prof = nullptr;  // optional sub-kernel timing
    long long h_pairs = 0;     // host copy of the current list size (kept while profiling)
    // partial-CCD filter: near list, double-buffered watch list, reference
    // displacement of the last full pass, bookkeeping
    long long cap_pairs = 0;
    DevBuf<int> near, watch[2];
    DevBuf<int> ccd_count;  // survivors of the full CCD's FP32 filter (listed in near)
    DevBuf<float4> disp0;
    DevBuf<PccdState> pccd;
    void reserve_pccd(const CollView &cv, cudaStream_t s);

    // superset lists of a hash pass with gap d_hat + 2 mu at positions (ref0,
    // ref1); while every vertex stays within mu' = 0.9 mu of that swept box,
    // the exact lists are a subsequence of them (see filter)
    DevBuf<int2> sup_vt, sup_ee;
    DevBuf<long long> sup_cnt;  // [2]
    DevBuf<float4> ref0, ref1;
    DevBuf<int> flags, fpos, fscratch;
    DevBuf<int> reuse_bad;
    float sup_mu = 0.f;
    bool sup_ok = false;

    // (re)allocates every buffer for the topology cv; the counts and the
    // partial-CCD state are reset on stream s
    void reserve(const CollView &cv, long long cap_vt, long long cap_ee, long long cap_ent, cudaStream_t s);
    // larger capacities keeping the current candidate lists, states and counts
    void grow(const CollView &cv, long long cap_vt, long long cap_ee, long long cap_ent, cudaStream_t s);
    void grow_slots(const CollView &cv, bool vt, bool ee);
    void run(cudaStream_t s, const CollView &cv, const float4 *x0, const float4 *x1, float dhat, int *overflow);
    // hash pass into the superset lists (gap dhat + 2 mu), then filter
    void run_super(cudaStream_t s, const CollView &cv, const float4 *x0, const float4 *x1, float dhat, float mu,
                   int *overflow);
    // true when every vertex of (x0, x1) lies in the reference swept box +- 0.9 mu (host sync)
    bool can_reuse(cudaStream_t s, const CollView &cv, const float4 *x0, const float4 *x1);
    // exact lists for (x0, x1) with gap dhat from the superset; makes them current
    void filter(cudaStream_t s, const CollView &cv, const float4 *x0, const float4 *x1, float dhat);
    // the hash pipeline writing into the given lists
    void hash_pass(cudaStream_t s, const CollView &cv, const float4 *x0, const float4 *x1, float dhat, int *overflow,
                   int2 *out_vt, int2 *out_ee, long long *out_nvt, long long *out_nee, int slot);
};

// Exact CCD over the current lists; if merge, NDB states are carried over
// from the previous lists (binary search by pair key), else start inactive.
// Pairs with an impact in [0,1] become active.  toi_min: atomic min (double bits).
void launch_full_ccd(cudaStream_t s, const CollView &cv, BroadPhase &bp, const float4 *x0, const float4 *x1,
                     const CollParams &P, bool merge, unsigned long long *toi_min);
// Rebuild the active list from the current states (closest points on xm).
void launch_collect_active(cudaStream_t s, const CollView &cv, BroadPhase &bp, const float4 *xm,
                           const CollParams &P, ActivePair *act, int cap_act, int *n_act, int *overflow);
// Partial CCD over (xm, xp) on the current lists: update states, rebuild the active list.
// disp (scratch, nv float4) receives xp - xm per collision vertex.
void launch_partial_ccd(cudaStream_t s, const CollView &cv, BroadPhase &bp, const float4 *xm, const float4 *xp,
                        const CollParams &P, ActivePair *act, int cap_act, int *n_act, int *overflow, float4 *disp);
// Collision springs of the active list at positions x: cw += w, cf += w (y - x).
// sets the weight of every listed active pair to k (residual forwarding, a = 0)
void launch_rf_weights(cudaStream_t s, ActivePair *act, const int *n_act, int cap_act, float k);
void launch_contact(cudaStream_t s, const CollView &cv, const ActivePair *act, const int *n_act, int cap_act,
                    const float4 *x, float dhat, float *cw, float4 *cf);
// Reads and clears (stream-ordered on s) the handle's index-guard word of the
// pair kernels (0: no entry of a pair, watch, near or active list pointed
// outside the topology).
unsigned int pair_guard_take(cudaStream_t s, unsigned int *guard);
// Compact the cloth vertices with cw > 0.
// (zero = false: *count has been zeroed already)
void launch_contact_list(cudaStream_t s, int n, const float *cw, int *list, int *count, const int *live = nullptr,
                         bool zero = true);

// Stage helpers on explicit quads (kinds: 0 VT, 1 EE).
void launch_ccd_quads(cudaStream_t s, const int4 *quads, const int *kinds, long long np, const float4 *x0,
                      const float4 *x1, double eta, double *toi);
void launch_partial_quads(cudaStream_t s, const int4 *quads, const int *kinds, long long np, const float4 *x0,
                          const float4 *x1, const CollParams &P, int *active);
void launch_activate_quads(cudaStream_t s, const int4 *quads, const int *kinds, const float *w, long long np,
                           const float4 *xm, ActivePair *act, int *n_act);
// Broad-phase lists as vertex quads for the stage entry point.
void launch_pairs_to_quads(cudaStream_t s, const CollView &cv, const int2 *ee, long long nee, int4 *out);

}  // namespace pdc
