// Collision kernels: spatial-hash broad phase, exact CCD (FP32 distance
// filter + FP64 root isolation), partial CCD with the non-distance barrier
// life-span counters, and the collision springs of the global step.
//
// Primitive pairs (Sec. 4): vertex-triangle (VT) and edge-edge (EE).  The
// candidate set is defined by an FP32 swept-box predicate; the hash only
// culls, so the lists equal the brute-force definition.  Lists are built
// with a count pass, a prefix sum and a write pass, and every primary's
// segment is sorted by the secondary id: the pair lists come out sorted by
// (primary, secondary) and deterministic, which lets the NDB counters of
// one full CCD be carried to the next by binary search.
#include <cooperative_groups.h>
#include <cstring>

#include "pdc_collide.cuh"
#include "pdc_scan.cuh"

namespace pdc {
namespace cg = cooperative_groups;

namespace {

constexpr int CELL_BIAS = 1 << 20;
constexpr int MAX_CELLS_PER_PRIM = 1 << 15;

__device__ inline int cell1(float v, float inv) {
    float c = floorf(v * inv);
    c = fminf(fmaxf(c, (float)(-CELL_BIAS)), (float)(CELL_BIAS - 1));
    return (int)c;
}
__device__ inline int3 cellv(float3 p, float inv) { return make_int3(cell1(p.x, inv), cell1(p.y, inv), cell1(p.z, inv)); }
__device__ inline unsigned long long cell_key(int x, int y, int z) {
    return ((unsigned long long)(x + CELL_BIAS) << 42) | ((unsigned long long)(y + CELL_BIAS) << 21) |
           (unsigned long long)(z + CELL_BIAS);
}
__device__ inline unsigned int hash_key(unsigned long long k, unsigned int mask) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return (unsigned int)k & mask;
}

__device__ inline float3 fmin3(float3 a, float3 b) { return make_float3(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z)); }
__device__ inline float3 fmax3(float3 a, float3 b) { return make_float3(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z)); }

// Candidate predicate: lo_a <= fl32(hi_b + dhat) and lo_b <= fl32(hi_a + dhat) on every axis.
__device__ inline bool box_overlap(float3 alo, float3 ahi, float3 blo, float3 bhi, float d) {
    return alo.x <= __fadd_rn(bhi.x, d) && blo.x <= __fadd_rn(ahi.x, d) && alo.y <= __fadd_rn(bhi.y, d) &&
           blo.y <= __fadd_rn(ahi.y, d) && alo.z <= __fadd_rn(bhi.z, d) && blo.z <= __fadd_rn(ahi.z, d);
}

// Cells of the table side: the primitive's own box, not inflated.
__device__ inline void cell_range_raw(float3 lo, float3 hi, float inv, int3 &clo, int3 &chi) {
    clo = cellv(lo, inv);
    chi = cellv(hi, inv);
}

// Cells searched by a query box b: if a table box a satisfies the predicate
// with b, then a_lo <= fl32(b_hi + d) and a_hi >= b_lo - d - |a_hi + d| 2^-24
// (from b_lo <= fl32(a_hi + d)); the search range covers both bounds (the
// low end is lowered by a margin of 2^-20 (|b_lo| + d) that exceeds the
// rounding of fl32(a_hi + d) and of its own computation), and floor(v / cell)
// is monotone, so the raw cell range of a meets it.  Only the query side is
// inflated: the gap is counted once.
__device__ inline float low_search(float lo, float d) {
    float m = (fabsf(lo) + d) * 9.5367431640625e-07f;  // 2^-20
    return __fsub_rn(__fsub_rn(lo, d), m);
}
__device__ inline void cell_range_query(float3 lo, float3 hi, float d, float inv, int3 &clo, int3 &chi) {
    float3 l = make_float3(low_search(lo.x, d), low_search(lo.y, d), low_search(lo.z, d));
    float3 h = make_float3(__fadd_rn(hi.x, d), __fadd_rn(hi.y, d), __fadd_rn(hi.z, d));
    clo = cellv(l, inv);
    chi = cellv(h, inv);
}

// A table entry stores (primitive << 3) | lowx | lowy << 1 | lowz << 2,
// where low* says that the entry's cell is the lowest cell of the
// primitive's raw range along that axis.  A pair is reported only in the
// lowest cell common to the query range and the table range, max(q_lo,
// t_lo) per axis; at a cell c of the query range this holds iff, per axis,
// low* is set or c equals the query's lowest cell.
__device__ inline bool owner_cell(int flags, int x, int y, int z, int3 qlo) {
    return ((flags & 1) || x == qlo.x) && ((flags & 2) || y == qlo.y) && ((flags & 4) || z == qlo.z);
}

__device__ inline void vbox(const float4 *x0, const float4 *x1, int v, float3 &lo, float3 &hi) {
    float3 a = f3(x0[v]), b = f3(x1[v]);
    lo = fmin3(a, b);
    hi = fmax3(a, b);
}

template <int K> __device__ inline void prim_box(const float4 *x0, const float4 *x1, const int *ids, float3 &lo, float3 &hi) {
    vbox(x0, x1, ids[0], lo, hi);
    for (int k = 1; k < K; ++k) {
        float3 l, h;
        vbox(x0, x1, ids[k], l, h);
        lo = fmin3(lo, l);
        hi = fmax3(hi, h);
    }
}

// ------------------------------------------------------------------ boxes
__global__ void k_tri_boxes(CollView cv, const float4 *__restrict__ x0, const float4 *__restrict__ x1,
                            float4 *__restrict__ blo, float4 *__restrict__ bhi, GridParams *gp) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    float ext = 0.f;
    if (t < cv.nt) {
        int4 T = cv.tri[t];
        int ids[3] = {T.x, T.y, T.z};
        float3 lo, hi;
        prim_box<3>(x0, x1, ids, lo, hi);
        blo[t] = f4(lo);
        bhi[t] = f4(hi);
        ext = fmaxf(hi.x - lo.x, fmaxf(hi.y - lo.y, hi.z - lo.z));
    }
    for (int o = 16; o > 0; o >>= 1) ext += __shfl_xor_sync(0xffffffffu, ext, o);
    if ((threadIdx.x & 31) == 0 && ext > 0.f) atomicAdd(&gp->ext_sum, (double)ext);
}

__global__ void k_edge_boxes(CollView cv, const float4 *__restrict__ x0, const float4 *__restrict__ x1,
                             float4 *__restrict__ blo, float4 *__restrict__ bhi) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cv.ne) return;
    int2 E = cv.edge[e];
    int ids[2] = {E.x, E.y};
    float3 lo, hi;
    prim_box<2>(x0, x1, ids, lo, hi);
    blo[e] = f4(lo);
    bhi[e] = f4(hi);
}

__global__ void k_grid_params(GridParams *gp, int nt, float dhat, float scale) {
    double mean = nt > 0 ? gp->ext_sum / nt : 0.0;
    float cell = fmaxf((float)mean, 2.f * dhat);
    cell = fmaxf(cell, 1e-6f) * scale;
    gp->cell = cell;
    gp->inv_cell = 1.f / cell;
}

// ------------------------------------------------------------------ hash table
// mode 0: count per bucket; mode 1: fill entries.
__global__ void k_hash_insert(int np, const float4 *__restrict__ blo, const float4 *__restrict__ bhi,
                              const GridParams *gp, float dhat, unsigned int mask, int *__restrict__ bcnt,
                              const int *__restrict__ bstart, int *__restrict__ bfill,
                              unsigned long long *__restrict__ ekey, int *__restrict__ eprim, int mode,
                              const long long *total, long long cap, int *overflow) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    if (mode == 1 && *total > cap) return;
    float inv = gp->inv_cell;
    int3 lo, hi;
    cell_range_raw(f3(blo[p]), f3(bhi[p]), inv, lo, hi);
    long long ncell = (long long)(hi.x - lo.x + 1) * (hi.y - lo.y + 1) * (hi.z - lo.z + 1);
    if (ncell > MAX_CELLS_PER_PRIM) {
        if (mode == 0) atomicOr(overflow, OVF_CELLS);
        return;
    }
    for (int z = lo.z; z <= hi.z; ++z)
        for (int y = lo.y; y <= hi.y; ++y)
            for (int x = lo.x; x <= hi.x; ++x) {
                unsigned long long k = cell_key(x, y, z);
                unsigned int b = hash_key(k, mask);
                if (mode == 0) {
                    atomicAdd(&bcnt[b], 1);
                } else {
                    int pos = bstart[b] + atomicAdd(&bfill[b], 1);
                    ekey[pos] = k;
                    eprim[pos] = (p << 3) | (x == lo.x ? 1 : 0) | (y == lo.y ? 2 : 0) | (z == lo.z ? 4 : 0);
                }
            }
}

// ------------------------------------------------------------------ queries
// Queries.  Each primary collects its candidates, sorted by secondary id,
// in a fixed-width row of a slot buffer; the count is always exact, and a
// primary with more candidates than the row width flags OVF_SLOTS (the pass
// is then rerun with wider rows).  In the VT query QG lanes share one
// vertex and stride over the entries of each bucket of its cell range
// together (the lanes of a group run the same trip count), append through a
// group ballot and sort the row once at the end.
constexpr int QUERY_T = 128;
// lanes per vertex in the VT query: 4, 8 (default) or 16 (BroadPhase::qg_vt)

__device__ inline void slot_insert(int *row, int width, int c, int q) {
    if (c >= width) return;
    int j = c - 1;
    while (j >= 0 && row[j] > q) {
        row[j + 1] = row[j];
        --j;
    }
    row[j + 1] = q;
}

__device__ inline void sort_row(int *row, int c) {
    for (int i = 1; i < c; ++i) {
        int q = row[i], j = i - 1;
        while (j >= 0 && row[j] > q) {
            row[j + 1] = row[j];
            --j;
        }
        row[j + 1] = q;
    }
}

// VT: primary = vertex v (all collision vertices), secondary = triangle.
template <int QG>
__global__ void __launch_bounds__(QUERY_T) k_query_vt(CollView cv, const float4 *__restrict__ x0,
                                                      const float4 *__restrict__ x1, const float4 *__restrict__ tlo,
                                                      const float4 *__restrict__ thi, const GridParams *gp, float dhat, unsigned int mask,
                                                      const int *__restrict__ bcnt, const int *__restrict__ bstart,
                                                      const unsigned long long *__restrict__ ekey,
                                                      const int *__restrict__ eprim, int *__restrict__ cnt,
                                                      int *__restrict__ slots, int width,
                                                      const long long *hash_total, long long cap_ent, int *overflow) {
    auto grp = cg::tiled_partition<QG>(cg::this_thread_block());
    const int gl = (int)grp.thread_rank();
    const int v = (blockIdx.x * blockDim.x + threadIdx.x) / QG;
    if (v >= cv.nv) return;  // uniform per group
    if (*hash_total > cap_ent) {  // table not filled: produce nothing
        if (gl == 0) cnt[v] = 0;
        return;
    }
    float inv = gp->inv_cell;
    float3 lo, hi;
    vbox(x0, x1, v, lo, hi);
    int3 clo, chi;
    cell_range_query(lo, hi, dhat, inv, clo, chi);
    if ((long long)(chi.x - clo.x + 1) * (chi.y - clo.y + 1) * (chi.z - clo.z + 1) > MAX_CELLS_PER_PRIM) {
        if (gl == 0) {
            cnt[v] = 0;
            atomicOr(overflow, OVF_CELLS);
        }
        return;
    }
    const bool vfix = v >= cv.nc;
    int *row = slots + (size_t)v * width;
    int c = 0;
    for (int z = clo.z; z <= chi.z; ++z)
        for (int y = clo.y; y <= chi.y; ++y)
            for (int x = clo.x; x <= chi.x; ++x) {
                const unsigned long long k = cell_key(x, y, z);
                const unsigned int b = hash_key(k, mask);
                const int e0 = bstart[b], e1 = e0 + bcnt[b];
                for (int eb = e0; eb < e1; eb += QG) {
                    const int e = eb + gl;
                    bool cand = false;
                    int t = 0;
                    if (e < e1 && ekey[e] == k) {
                        const int pk = eprim[e];
                        t = pk >> 3;
                        if (owner_cell(pk, x, y, z, clo)) {
                            int4 T = cv.tri[t];
                            cand = T.x != v && T.y != v && T.z != v &&
                                   !(vfix && T.x >= cv.nc && T.y >= cv.nc && T.z >= cv.nc) &&
                                   box_overlap(lo, hi, f3(tlo[t]), f3(thi[t]), dhat);
                        }
                    }
                    const unsigned m = grp.ballot(cand);
                    if (cand) {
                        int slot = c + __popc(m & ((1u << gl) - 1u));
                        if (slot < width) row[slot] = t;
                    }
                    c += __popc(m);
                }
            }
    grp.sync();
    if (gl == 0) {
        sort_row(row, min(c, width));
        cnt[v] = c;
        if (c > width) atomicOr(overflow, OVF_SLOTS);
    }
}

// EE: primary = edge e, secondary = edge f > e; one thread per edge (the
// edge buckets are short and half their entries fail f > e at once, so the
// grouped scan of the VT query does not pay here: measured slower).
__global__ void __launch_bounds__(QUERY_T) k_query_ee(CollView cv, const float4 *__restrict__ elo,
                                                  const float4 *__restrict__ ehi, const GridParams *gp, float dhat, unsigned int mask,
                                                  const int *__restrict__ bcnt, const int *__restrict__ bstart,
                                                  const unsigned long long *__restrict__ ekey,
                                                  const int *__restrict__ eprim, int *__restrict__ cnt,
                                                  int *__restrict__ slots, int width,
                                                  const long long *hash_total, long long cap_ent, int *overflow) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cv.ne) return;
    if (*hash_total > cap_ent) {
        cnt[e] = 0;
        return;
    }
    float inv = gp->inv_cell;
    float3 lo = f3(elo[e]), hi = f3(ehi[e]);
    int3 clo, chi;
    cell_range_query(lo, hi, dhat, inv, clo, chi);
    if ((long long)(chi.x - clo.x + 1) * (chi.y - clo.y + 1) * (chi.z - clo.z + 1) > MAX_CELLS_PER_PRIM) {
        cnt[e] = 0;
        atomicOr(overflow, OVF_CELLS);
        return;
    }
    int2 E = cv.edge[e];
    bool efix = E.x >= cv.nc && E.y >= cv.nc;
    int *row = slots + (size_t)e * width;
    int c = 0;
    for (int z = clo.z; z <= chi.z; ++z)
        for (int y = clo.y; y <= chi.y; ++y)
            for (int x = clo.x; x <= chi.x; ++x) {
                unsigned long long k = cell_key(x, y, z);
                unsigned int b = hash_key(k, mask);
                int e0 = bstart[b], e1 = e0 + bcnt[b];
                for (int q = e0; q < e1; ++q) {
                    if (ekey[q] != k) continue;
                    const int pk = eprim[q];
                    const int f = pk >> 3;
                    if (f <= e) continue;
                    if (!owner_cell(pk, x, y, z, clo)) continue;
                    int2 F = cv.edge[f];
                    if (E.x == F.x || E.x == F.y || E.y == F.x || E.y == F.y) continue;
                    if (efix && F.x >= cv.nc && F.y >= cv.nc) continue;
                    if (!box_overlap(lo, hi, f3(elo[f]), f3(ehi[f]), dhat)) continue;
                    slot_insert(row, width, c, f);
                    ++c;
                }
            }
    cnt[e] = c;
    if (c > width) atomicOr(overflow, OVF_SLOTS);
}

// out[off[p] + k] = (p, slots[p][k]) for k < cnt[p]
__global__ void k_compact_slots(int np, const int *__restrict__ cnt, const int *__restrict__ off,
                                const int *__restrict__ slots, int width, const long long *total, long long cap,
                                int2 *__restrict__ out) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np || *total > cap) return;
    int c = min(cnt[p], width), o = off[p];
    const int *row = slots + (size_t)p * width;
    for (int k = 0; k < c; ++k) out[o + k] = make_int2(p, row[k]);
}

__global__ void k_check_cap(const long long *total, long long cap, int flag, int *overflow, long long *count_out) {
    long long t = *total;
    bool bad = t > cap || (*overflow & (OVF_SLOTS | OVF_CELLS | OVF_HASH)) != 0;
    *count_out = bad ? 0 : t;
    if (t > cap) atomicOr(overflow, flag);
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

// ====================================================================== broad phase driver
namespace {
__global__ void k_pccd_force(PccdState *ps) { ps->force_full = 1; }

// bad |= some coordinate of x0_v or x1_v leaves [min(r0,r1) - m, max(r0,r1) + m]
__global__ void k_containment(int nv, const float4 *__restrict__ x0, const float4 *__restrict__ x1,
                              const float4 *__restrict__ r0, const float4 *__restrict__ r1, float m, int *bad) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    float3 a = f3(r0[v]), b = f3(r1[v]);
    float3 lo = make_float3(fminf(a.x, b.x) - m, fminf(a.y, b.y) - m, fminf(a.z, b.z) - m);
    float3 hi = make_float3(fmaxf(a.x, b.x) + m, fmaxf(a.y, b.y) + m, fmaxf(a.z, b.z) + m);
    float3 p = f3(x0[v]), q = f3(x1[v]);
    bool in = p.x >= lo.x && p.y >= lo.y && p.z >= lo.z && p.x <= hi.x && p.y <= hi.y && p.z <= hi.z &&
              q.x >= lo.x && q.y >= lo.y && q.z >= lo.z && q.x <= hi.x && q.y <= hi.y && q.z <= hi.z;
    if (!in) atomicOr(bad, 1);
}

// flag[i] = pair i of a superset list passes the broad-phase predicate on the
// current boxes (kind 0: (v, t) with the vertex's swept box; 1: (e, f))
__global__ void k_pair_flags(int kind, int n, const int2 *__restrict__ list, const float4 *__restrict__ x0,
                             const float4 *__restrict__ x1, const float4 *__restrict__ tlo,
                             const float4 *__restrict__ thi, const float4 *__restrict__ elo,
                             const float4 *__restrict__ ehi, float dhat, int *__restrict__ flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int2 p = list[i];
    float3 alo, ahi, blo, bhi;
    if (kind == 0) {
        vbox(x0, x1, p.x, alo, ahi);
        blo = f3(tlo[p.y]);
        bhi = f3(thi[p.y]);
    } else {
        alo = f3(elo[p.x]);
        ahi = f3(ehi[p.x]);
        blo = f3(elo[p.y]);
        bhi = f3(ehi[p.y]);
    }
    flag[i] = box_overlap(alo, ahi, blo, bhi, dhat) ? 1 : 0;
}

__global__ void k_pair_scatter(int n, const int2 *__restrict__ list, const int *__restrict__ flag,
                               const int *__restrict__ pos, int2 *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i]] = list[i];
}
}  // namespace

void BroadPhase::reserve(const CollView &cv, long long cap_vt_, long long cap_ee_, long long cap_ent_,
                         cudaStream_t s) {
    ++gen;
    nt = cv.nt;
    ne = cv.ne;
    nv = cv.nv;
    auto pow2 = [](long long x) {
        long long p = 1024;
        while (p < x) p <<= 1;
        return p;
    };
    T_vt = (int)pow2(2LL * cv.nt + 1024);
    T_ee = (int)pow2(2LL * cv.ne + 1024);
    for (int k = 0; k < 2; ++k) {
        bcnt[k].alloc(k == 0 ? T_vt : T_ee);
        bstart[k].alloc(k == 0 ? T_vt : T_ee);
        bfill[k].alloc(k == 0 ? T_vt : T_ee);
    }
    cap_ent = cap_ent_;
    for (int k = 0; k < 2; ++k) {
        ekey[k].alloc(cap_ent);
        eprim[k].alloc(cap_ent);
    }
    tlo.alloc(cv.nt);
    thi.alloc(cv.nt);
    elo.alloc(cv.ne);
    ehi.alloc(cv.ne);
    cnt_v.alloc(cv.nv);
    off_v.alloc(cv.nv);
    cnt_e.alloc(cv.ne);
    off_e.alloc(cv.ne);
    if (cv.nt >= (1 << 28) || cv.ne >= (1 << 28))
        throw Error(PDC_ERR_ARG, "broad phase: more than 2^28 triangles or edges");
    slots_vt.alloc((size_t)cv.nv * w_vt);
    slots_ee.alloc((size_t)cv.ne * w_ee);
    long long mx = std::max<long long>(std::max<long long>(T_vt, T_ee), std::max<long long>(cv.nv, cv.ne));
    scratch.alloc(scan_scratch_ints((int)mx) + 16);
    gp.alloc(1);
    totals.alloc(8);
    cap_vt = cap_vt_;
    cap_ee = cap_ee_;
    for (int k = 0; k < 2; ++k) {
        vt[k].alloc(cap_vt);
        ee[k].alloc(cap_ee);
        st_vt[k].alloc(cap_vt);
        st_ee[k].alloc(cap_ee);
        d0_vt[k].alloc(cap_vt);
        d0_ee[k].alloc(cap_ee);
        cnt_vt_d[k].alloc(1);
        cnt_ee_d[k].alloc(1);
    }
    cur = 0;
    sup_ok = false;
    for (int k = 0; k < 2; ++k) {
        cnt_vt_d[k].zero(s);
        cnt_ee_d[k].zero(s);
    }
    reserve_pccd(cv, s);
}

void BroadPhase::reserve_pccd(const CollView &cv, cudaStream_t s) {
    ++gen;
    cap_pairs = cap_vt + cap_ee;
    near.alloc(cap_pairs);
    watch[0].alloc(cap_pairs);
    watch[1].alloc(cap_pairs);
    disp0.alloc(std::max(cv.nv, 1));
    disp0.zero(s);
    pccd.alloc(1);
    pccd.zero(s);  // no watch list yet: the first pass scans every pair
    k_pccd_force<<<1, 1, 0, s>>>(pccd);
    PDC_LAUNCH_CK();
}

template <class T> static void grow_keep(DevBuf<T> &b, long long cap, cudaStream_t s) {
    if ((long long)b.n >= cap) return;
    DevBuf<T> nb;
    nb.alloc(cap);
    if (b.p && b.n) PDC_CK(cudaMemcpyAsync(nb.p, b.p, sizeof(T) * b.n, cudaMemcpyDeviceToDevice, s));
    PDC_CK(cudaStreamSynchronize(s));
    std::swap(b.p, nb.p);
    std::swap(b.n, nb.n);
}

void BroadPhase::grow_slots(const CollView &cv, bool vt_, bool ee_) {
    if (vt_) {
        w_vt *= 2;
        slots_vt.alloc((size_t)cv.nv * w_vt);
    }
    if (ee_) {
        w_ee *= 2;
        slots_ee.alloc((size_t)cv.ne * w_ee);
    }
}

void BroadPhase::grow(const CollView &cv, long long cvt, long long cee, long long cent, cudaStream_t s) {
    ++gen;
    if (cent > cap_ent) {
        cap_ent = cent;
        for (int k = 0; k < 2; ++k) {
            ekey[k].alloc(cap_ent);
            eprim[k].alloc(cap_ent);
        }
    }
    if (cvt > cap_vt) {
        cap_vt = cvt;
        for (int k = 0; k < 2; ++k) {
            grow_keep(vt[k], cap_vt, s);
            grow_keep(st_vt[k], cap_vt, s);
            grow_keep(d0_vt[k], cap_vt, s);
        }
    }
    if (cee > cap_ee) {
        cap_ee = cee;
        for (int k = 0; k < 2; ++k) {
            grow_keep(ee[k], cap_ee, s);
            grow_keep(st_ee[k], cap_ee, s);
            grow_keep(d0_ee[k], cap_ee, s);
        }
    }
    if (cap_vt + cap_ee > cap_pairs) {
        PDC_CK(cudaStreamSynchronize(s));
        reserve_pccd(cv, s);
    }
}

// Builds the new candidate lists in buffer (cur ^ 1) and makes it current.
#define BP_PROF(name, ...)                                                                            \
    do {                                                                                               \
        if (prof) prof->begin(s, name, 0.0);                                                           \
        __VA_ARGS__;                                                                                   \
        if (prof) prof->end(s);                                                                        \
    } while (0)

void BroadPhase::run(cudaStream_t s, const CollView &cv, const float4 *x0, const float4 *x1, float dhat,
                     int *overflow) {
    int nw = cur ^ 1;
    hash_pass(s, cv, x0, x1, dhat, overflow, vt[nw], ee[nw], cnt_vt_d[nw], cnt_ee_d[nw]);
    cur = nw;
    sup_ok = false;
    k_pccd_force<<<1, 1, 0, s>>>(pccd);  // new lists: the next partial-CCD pass scans them all
    PDC_LAUNCH_CK();
}

void BroadPhase::hash_pass(cudaStream_t s, const CollView &cv, const float4 *x0, const float4 *x1, float dhat,
                           int *overflow, int2 *out_vt, int2 *out_ee, long long *out_nvt, long long *out_nee) {
    PDC_CK(cudaMemsetAsync(gp.p, 0, sizeof(GridParams), s));
    BP_PROF("bp_boxes", if (cv.nt) k_tri_boxes<<<nblk(cv.nt, 256), 256, 0, s>>>(cv, x0, x1, tlo, thi, gp);
            if (cv.ne) k_edge_boxes<<<nblk(cv.ne, 256), 256, 0, s>>>(cv, x0, x1, elo, ehi);
            k_grid_params<<<1, 1, 0, s>>>(gp, cv.nt, dhat, cell_scale));
    PDC_LAUNCH_CK();
    long long *tot = totals.p;
    // ---- tables: 0 = triangles (VT), 1 = edges (EE)
    for (int k = 0; k < 2; ++k) {
        int np = k == 0 ? cv.nt : cv.ne;
        int T = k == 0 ? T_vt : T_ee;
        const float4 *lo = k == 0 ? tlo.p : elo.p;
        const float4 *hi = k == 0 ? thi.p : ehi.p;
        BP_PROF("bp_hash_build", bcnt[k].zero(s); bfill[k].zero(s);
        if (np) {
            k_hash_insert<<<nblk(np, 256), 256, 0, s>>>(np, lo, hi, gp, dhat, (unsigned)(T - 1), bcnt[k], bstart[k],
                                                        bfill[k], ekey[k], eprim[k], 0, tot + k, cap_ent, overflow);
            PDC_LAUNCH_CK();
        }
        exclusive_scan(s, bcnt[k], bstart[k], T, scratch, tot + k);
        k_check_cap<<<1, 1, 0, s>>>(tot + k, cap_ent, OVF_HASH, overflow, tot + 4 + k);
        if (np) {
            k_hash_insert<<<nblk(np, 256), 256, 0, s>>>(np, lo, hi, gp, dhat, (unsigned)(T - 1), bcnt[k], bstart[k],
                                                        bfill[k], ekey[k], eprim[k], 1, tot + k, cap_ent, overflow);
            PDC_LAUNCH_CK();
        });
    }
    // ---- VT candidates
    if (prof) prof->begin(s, "bp_query_vt", 0.0);
    if (cv.nv) {
        auto query = [&](int qg) {
#define PDC_QVT(Q)                                                                                                   \
    k_query_vt<Q><<<nblk((long long)cv.nv * Q, QUERY_T), QUERY_T, 0, s>>>(cv, x0, x1, tlo, thi, gp, dhat,             \
                                                                          (unsigned)(T_vt - 1), bcnt[0], bstart[0],  \
                                                                          ekey[0], eprim[0], cnt_v, slots_vt, w_vt,  \
                                                                          tot + 0, cap_ent, overflow)
            if (qg == 4) PDC_QVT(4);
            else if (qg == 16) PDC_QVT(16);
            else PDC_QVT(8);
#undef PDC_QVT
            PDC_LAUNCH_CK();
        };
        if (tune_query) {
            // each candidate writes the same counts and rows: time each, keep the fastest
            tune_query = false;
            const int cand[3] = {4, 8, 16};
            cudaEvent_t e[4];
            for (auto &ev : e) PDC_CK(cudaEventCreate(&ev));
            query(8);  // warm-up
            PDC_CK(cudaEventRecord(e[0], s));
            for (int k = 0; k < 3; ++k) {
                query(cand[k]);
                PDC_CK(cudaEventRecord(e[k + 1], s));
            }
            PDC_CK(cudaEventSynchronize(e[3]));
            int best = 1;
            for (int k = 0; k < 3; ++k) {
                PDC_CK(cudaEventElapsedTime(&query_ms[k], e[k], e[k + 1]));
                if (query_ms[k] < query_ms[best]) best = k;
            }
            for (auto &ev : e) cudaEventDestroy(ev);
            qg_vt = cand[best];
        }
        query(qg_vt);
    }
    exclusive_scan(s, cnt_v, off_v, cv.nv, scratch, tot + 2);
    k_check_cap<<<1, 1, 0, s>>>(tot + 2, cap_vt, OVF_VT, overflow, out_nvt);
    if (cv.nv) {
        k_compact_slots<<<nblk(cv.nv, 256), 256, 0, s>>>(cv.nv, cnt_v, off_v, slots_vt, w_vt, tot + 2, cap_vt, out_vt);
        PDC_LAUNCH_CK();
    }
    if (prof) prof->end(s);
    // ---- EE candidates
    if (prof) prof->begin(s, "bp_query_ee", 0.0);
    if (cv.ne) {
        k_query_ee<<<nblk(cv.ne, QUERY_T), QUERY_T, 0, s>>>(
            cv, elo, ehi, gp, dhat, (unsigned)(T_ee - 1), bcnt[1], bstart[1], ekey[1], eprim[1], cnt_e,
            slots_ee, w_ee, tot + 1, cap_ent, overflow);
        PDC_LAUNCH_CK();
    }
    exclusive_scan(s, cnt_e, off_e, cv.ne, scratch, tot + 3);
    k_check_cap<<<1, 1, 0, s>>>(tot + 3, cap_ee, OVF_EE, overflow, out_nee);
    if (cv.ne) {
        k_compact_slots<<<nblk(cv.ne, 256), 256, 0, s>>>(cv.ne, cnt_e, off_e, slots_ee, w_ee, tot + 3, cap_ee, out_ee);
        PDC_LAUNCH_CK();
    }
    if (prof) prof->end(s);
}

void BroadPhase::run_super(cudaStream_t s, const CollView &cv, const float4 *x0, const float4 *x1, float dhat,
                           float mu, int *overflow) {
    if (sup_vt.n < (size_t)cap_vt) sup_vt.alloc(cap_vt);
    if (sup_ee.n < (size_t)cap_ee) sup_ee.alloc(cap_ee);
    sup_cnt.alloc(2);
    // gap of the superset: every pair within d_hat of each other on a swept
    // box grown by mu' per side is within d_hat + 2 mu on the reference boxes
    float gap = dhat + 2.f * mu;
    hash_pass(s, cv, x0, x1, gap, overflow, sup_vt, sup_ee, sup_cnt.p, sup_cnt.p + 1);
    long long cnt[2] = {0, 0};
    sup_cnt.download(cnt, 2, s);
    PDC_CK(cudaStreamSynchronize(s));
    if (std::max(cnt[0], cnt[1]) > scan_capacity()) {  // too long to filter: plain pass
        run(s, cv, x0, x1, dhat, overflow);
        return;
    }
    ref0.alloc(std::max(cv.nv, 1));
    ref1.alloc(std::max(cv.nv, 1));
    if (cv.nv) {
        PDC_CK(cudaMemcpyAsync(ref0.p, x0, sizeof(float4) * cv.nv, cudaMemcpyDeviceToDevice, s));
        PDC_CK(cudaMemcpyAsync(ref1.p, x1, sizeof(float4) * cv.nv, cudaMemcpyDeviceToDevice, s));
    }
    sup_mu = mu;
    filter(s, cv, x0, x1, dhat);
    sup_ok = true;
}

bool BroadPhase::can_reuse(cudaStream_t s, const CollView &cv, const float4 *x0, const float4 *x1) {
    if (!sup_ok || cv.nv != nv) return false;
    reuse_bad.alloc(1);
    reuse_bad.zero(s);
    if (cv.nv) k_containment<<<nblk(cv.nv, 256), 256, 0, s>>>(cv.nv, x0, x1, ref0, ref1, 0.9f * sup_mu, reuse_bad);
    PDC_LAUNCH_CK();
    int bad = 1;
    reuse_bad.download(&bad, 1, s);
    PDC_CK(cudaStreamSynchronize(s));
    return bad == 0;
}

void BroadPhase::filter(cudaStream_t s, const CollView &cv, const float4 *x0, const float4 *x1, float dhat) {
    int nw = cur ^ 1;
    long long cnt[2] = {0, 0};
    sup_cnt.download(cnt, 2, s);
    PDC_CK(cudaStreamSynchronize(s));
    long long mx = std::max<long long>(std::max(cnt[0], cnt[1]), 1);
    if (mx > scan_capacity()) throw Error(PDC_ERR_CAPACITY, "superset list too long to filter");
    if ((long long)flags.n < mx) {
        flags.alloc(mx);
        fpos.alloc(mx);
        fscratch.alloc(scan_scratch_ints((int)mx) + 16);
    }
    if (prof) prof->begin(s, "bp_filter", 0.0);
    // boxes over the new interval, with the same arithmetic as the hash pass
    if (cv.nt) k_tri_boxes<<<nblk(cv.nt, 256), 256, 0, s>>>(cv, x0, x1, tlo, thi, gp);
    if (cv.ne) k_edge_boxes<<<nblk(cv.ne, 256), 256, 0, s>>>(cv, x0, x1, elo, ehi);
    PDC_LAUNCH_CK();
    long long *tot = totals.p;
    for (int k = 0; k < 2; ++k) {
        int n = (int)cnt[k];
        const int2 *in = k == 0 ? sup_vt.p : sup_ee.p;
        int2 *out = k == 0 ? vt[nw].p : ee[nw].p;
        long long *nout = k == 0 ? cnt_vt_d[nw].p : cnt_ee_d[nw].p;
        if (n > 0) {
            k_pair_flags<<<nblk(n, 256), 256, 0, s>>>(k, n, in, x0, x1, tlo, thi, elo, ehi, dhat, flags);
            PDC_LAUNCH_CK();
        }
        exclusive_scan(s, flags, fpos, n, fscratch, tot + 6 + k);
        if (n > 0) {
            k_pair_scatter<<<nblk(n, 256), 256, 0, s>>>(n, in, flags, fpos, out);
            PDC_LAUNCH_CK();
        }
        PDC_CK(cudaMemcpyAsync(nout, tot + 6 + k, sizeof(long long), cudaMemcpyDeviceToDevice, s));
    }
    if (prof) prof->end(s);
    cur = nw;
    k_pccd_force<<<1, 1, 0, s>>>(pccd);  // new lists: the next partial-CCD pass scans them all
    PDC_LAUNCH_CK();
}

}  // namespace pdc
