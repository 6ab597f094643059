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
__device__ inline int3 cellv(float3 p, float3 inv) {
    return make_int3(cell1(p.x, inv.x), cell1(p.y, inv.y), cell1(p.z, inv.z));
}
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
    float3 ext = make_float3(0.f, 0.f, 0.f);
    if (t < cv.nt) {
        int4 T = cv.tri[t];
        int ids[3] = {T.x, T.y, T.z};
        float3 lo, hi;
        prim_box<3>(x0, x1, ids, lo, hi);
        blo[t] = f4(lo);
        bhi[t] = f4(hi);
        ext = hi - lo;
    }
    // per-axis sums: warp, then block (one atomic per axis and block)
    __shared__ float part[3][32];
    for (int o = 16; o > 0; o >>= 1) {
        ext.x += __shfl_xor_sync(0xffffffffu, ext.x, o);
        ext.y += __shfl_xor_sync(0xffffffffu, ext.y, o);
        ext.z += __shfl_xor_sync(0xffffffffu, ext.z, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        part[0][w] = ext.x;
        part[1][w] = ext.y;
        part[2][w] = ext.z;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double sum = 0.0;
        for (int k = 0; k < nw; ++k) sum += part[threadIdx.x][k];
        if (sum > 0.0) atomicAdd(&gp->ext_sum[threadIdx.x], sum);
    }
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
    for (int d = 0; d < 3; ++d) {
        double mean = nt > 0 ? gp->ext_sum[d] / nt : 0.0;
        float cell = fmaxf((float)mean, 2.f * dhat);
        cell = fmaxf(cell, 1e-6f) * scale;
        gp->cell[d] = cell;
        gp->inv_cell[d] = 1.f / cell;
    }
}

constexpr int CELL_CHUNK = 64;
constexpr unsigned FL_FIXED = 1u << 3;       // every vertex of the primitive is an obstacle vertex
constexpr unsigned Q_GUARD = (1u << 8) | (1u << 17) | (1u << 26);
constexpr unsigned Q_OWNER = 7u << 27;       // lowest-cell flags in the low corner's word
constexpr unsigned Q_FIXED = FL_FIXED << 27;
constexpr int QUEUE = 64;                    // survivor queue per warp

__device__ inline unsigned quant_lo(float v, float c0, float s) {
    return (unsigned)fminf(fmaxf(floorf(__fmul_rn(__fsub_rn(v, c0), s)), 0.f), 255.f);
}
__device__ inline unsigned quant_hi(float v, float c0, float s) {
    return (unsigned)fminf(fmaxf(ceilf(__fmul_rn(__fsub_rn(v, c0), s)), 0.f), 255.f);
}

// ------------------------------------------------------------------ cell table
// Table primitives: collision vertices [0, nv), edges [nv, nv + ne),
// triangles [nv + ne, nv + ne + nt).  Primitive p covers the cells of its
// swept box with the upper side raised by d_hat, [lo, fl32(hi + d_hat)].  Two
// raised boxes overlap on an axis iff lo_a <= fl32(hi_b + d) and lo_b <=
// fl32(hi_a + d), which is the candidate predicate itself; then the cell of
// max(lo_a, lo_b) per axis lies in both cell ranges (floor(v / cell) is
// monotone), and it is the one common cell where, per axis, one of the two
// entries sits at the lowest cell of its range (the owner test below), so
// every candidate pair is tested in exactly one cell.
constexpr int KIND_V = 0, KIND_E = 1, KIND_T = 2;
constexpr unsigned PAY_PRIM = (1u << 27) - 1;

__device__ inline unsigned pay_pack(int prim, int kind, int low) {
    return (unsigned)prim | ((unsigned)kind << 27) | ((unsigned)low << 29);
}

__device__ inline float3 raise_d(float3 h, float d) {
    return make_float3(__fadd_rn(h.x, d), __fadd_rn(h.y, d), __fadd_rn(h.z, d));
}

// The swept box of table primitive p (not raised), its kind and id.
__device__ inline void table_box(const CollView &cv, const float4 *x0, const float4 *x1, const float4 *tlo,
                                 const float4 *thi, const float4 *elo, const float4 *ehi, int p, int &kind,
                                 int &prim, float3 &lo, float3 &hi) {
    if (p < cv.nv) {
        kind = KIND_V;
        prim = p;
        vbox(x0, x1, p, lo, hi);
    } else if (p < cv.nv + cv.ne) {
        kind = KIND_E;
        prim = p - cv.nv;
        lo = f3(elo[prim]);
        hi = f3(ehi[prim]);
    } else {
        kind = KIND_T;
        prim = p - cv.nv - cv.ne;
        lo = f3(tlo[prim]);
        hi = f3(thi[prim]);
    }
}

// mode 0: count the entries of every bucket; mode 1: write them.  In each
// round every lane takes the next cell of its primitive, and the lanes that
// land in the same bucket are served by one atomic (match_any), so
// neighbouring primitives (the mesh order is spatially coherent) share it.
__global__ void k_cell_insert(CollView cv, const float4 *__restrict__ x0, const float4 *__restrict__ x1,
                              const float4 *__restrict__ tlo, const float4 *__restrict__ thi,
                              const float4 *__restrict__ elo, const float4 *__restrict__ ehi, const GridParams *gp,
                              float dhat, unsigned int mask, int *__restrict__ bcnt, const int *__restrict__ bstart,
                              int *__restrict__ bfill, unsigned long long *__restrict__ ekey,
                              unsigned int *__restrict__ epay, unsigned long long *__restrict__ equ, int mode,
                              const long long *total, long long cap, int *overflow) {
    const int np = cv.nv + cv.ne + cv.nt;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned lane = threadIdx.x & 31;
    if (mode == 1 && *total > cap) return;  // the table does not fit (uniform over the grid)
    const float3 inv = make_float3(gp->inv_cell[0], gp->inv_cell[1], gp->inv_cell[2]);
    int kind = 0, prim = 0, ncell = 0;
    int3 lo = make_int3(0, 0, 0), hi = make_int3(-1, -1, -1);
    float3 l = make_float3(0.f, 0.f, 0.f), h = l;
    if (p < np) {
        table_box(cv, x0, x1, tlo, thi, elo, ehi, p, kind, prim, l, h);
        lo = cellv(l, inv);
        hi = cellv(raise_d(h, dhat), inv);
        long long nc = (long long)(hi.x - lo.x + 1) * (hi.y - lo.y + 1) * (hi.z - lo.z + 1);
        if (nc > MAX_CELLS_PER_PRIM) {
            if (mode == 0) atomicOr(overflow, OVF_CELLS);
        } else {
            ncell = (int)nc;
        }
    }
    const int sx = hi.x - lo.x + 1, sy = hi.y - lo.y + 1;
    const int rounds = __reduce_max_sync(0xffffffffu, (unsigned)ncell);
    // fill pass: the raised box, the kinematic flag and the quantization scale
    unsigned fixed = 0;
    float3 hr = h, qs = make_float3(0.f, 0.f, 0.f);
    if (mode == 1 && ncell > 0) {
        hr = raise_d(h, dhat);
        qs = make_float3(256.f / gp->cell[0], 256.f / gp->cell[1], 256.f / gp->cell[2]);
        if (kind == KIND_V) fixed = prim >= cv.nc;
        else if (kind == KIND_E) {
            const int2 E = cv.edge[prim];
            fixed = E.x >= cv.nc && E.y >= cv.nc;
        } else {
            const int4 Tr = cv.tri[prim];
            fixed = Tr.x >= cv.nc && Tr.y >= cv.nc && Tr.z >= cv.nc;
        }
    }
    for (int r = 0; r < rounds; ++r) {
        const bool act = r < ncell;
        int x = 0, y = 0, z = 0;
        unsigned long long k = 0;
        unsigned int b = 0xffffffffu;  // no bucket (mask < 2^31)
        if (act) {
            x = lo.x + r % sx;
            y = lo.y + (r / sx) % sy;
            z = lo.z + r / (sx * sy);
            k = cell_key(x, y, z);
            b = hash_key(k, mask);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        if (!act) continue;
        const int leader = __ffs(peers) - 1;
        if (mode == 0) {
            if ((int)lane == leader) atomicAdd(&bcnt[b], __popc(peers));
        } else {
            int base = 0;
            if ((int)lane == leader) base = atomicAdd(&bfill[b], __popc(peers));
            base = __shfl_sync(peers, base, leader);
            const int pos = bstart[b] + base + __popc(peers & ((1u << lane) - 1u));
            const unsigned low = (x == lo.x ? 1u : 0u) | (y == lo.y ? 2u : 0u) | (z == lo.z ? 4u : 0u);
            ekey[pos] = k;
            epay[pos] = pay_pack(prim, kind, (int)low);
            // the box quantized within this cell (cell origin from its index)
            const float cx = __fmul_rn((float)x, gp->cell[0]), cy = __fmul_rn((float)y, gp->cell[1]),
                        cz = __fmul_rn((float)z, gp->cell[2]);
            const unsigned ql = quant_lo(l.x, cx, qs.x) | (quant_lo(l.y, cy, qs.y) << 9) |
                                (quant_lo(l.z, cz, qs.z) << 18) | ((low | (fixed ? FL_FIXED : 0u)) << 27);
            const unsigned qh = quant_hi(hr.x, cx, qs.x) | (quant_hi(hr.y, cy, qs.y) << 9) |
                                (quant_hi(hr.z, cz, qs.z) << 18) | Q_GUARD;
            equ[pos] = (unsigned long long)ql | ((unsigned long long)qh << 32);
        }
    }
}

// ------------------------------------------------------------------ cell pairs
// A warp takes buckets 32 at a time from a global counter and, for every
// bucket with two entries or more, loads its entries into shared memory in
// chunks of CELL_CHUNK (boxes, vertex ids, cell keys, lists per kind) and
// tests every VT pair and every unordered EE pair of each chunk and of each
// pair of chunks, lanes striding over the flattened pair index.  Entries of
// other cells that share the bucket are told apart by their keys.  A
// candidate (v, t) or (e, f), e < f, is appended to the row of v or e; rows
// are sorted when they are compacted.
//
// Most pairs that share a cell fail either the owner test or the predicate,
// so each entry also carries its raised box quantized to 8 bits per axis
// within the cell, q = clamp(floor or ceil((v - cell origin) * 256 / cell),
// 0, 255): a map that is monotone in v, so quantized boxes of a pair that
// meets the predicate in this cell meet too.  The three fields sit at bits
// 0, 9 and 18 of a word, the high corner's word with the guard bits 8, 17
// and 26 set, so that one subtraction compares all three (a field's guard
// bit survives hi - lo iff lo <= hi); the low corner's word carries the
// owner flags (bits 27..29) and FL_FIXED (bit 30).  Pairs that pass this
// prefilter go through a per-warp queue to the full test, so that the rare
// survivors do not stall the lanes that keep scanning.
// One chunk of a bucket in shared memory, in kind order: vertices [0, nv),
// edges [nv, nv + ne), triangles [nv + ne, nv + ne + nt): cell key,
// quantized box words (as the insert pass wrote them) and primitive id.  The
// exact boxes and vertex ids of a pair are read from device memory only for
// the pairs that pass the prefilter.
struct CellRegion {
    unsigned long long key[CELL_CHUNK];
    unsigned int qlo[CELL_CHUNK];  // quantized low corner | (lowest-cell flags | FL_FIXED) << 27
    unsigned int qhi[CELL_CHUNK];  // quantized raised high corner | Q_GUARD
    int pid[CELL_CHUNK];
};

// per warp: two chunk regions and the survivor queue
struct CellWarp {
    CellRegion r[2];
    unsigned int queue[QUEUE];
};

struct KindCounts {
    int v, e, t;
};

// Loads entries [e0, e0 + cnt) of the table into R in kind order (a count
// pass over the payloads, then the write pass); coalesced, no gathers.
__device__ __forceinline__ KindCounts load_chunk(CellRegion &R, const unsigned long long *ekey,
                                                 const unsigned int *epay, const unsigned long long *equ, int e0,
                                                 int cnt, unsigned lane) {
    const unsigned below = (1u << lane) - 1u;
    KindCounts kc = {0, 0, 0};
    for (int base = 0; base < cnt; base += 32) {  // warp-uniform
        const int i = base + (int)lane;
        const int kind = i < cnt ? (int)((epay[e0 + i] >> 27) & 3u) : -1;
        kc.v += __popc(__ballot_sync(0xffffffffu, kind == KIND_V));
        kc.e += __popc(__ballot_sync(0xffffffffu, kind == KIND_E));
        kc.t += __popc(__ballot_sync(0xffffffffu, kind == KIND_T));
    }
    int cv_ = 0, ce = kc.v, ct = kc.v + kc.e;  // next slot of each kind
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + (int)lane;
        unsigned pay = 0;
        int kind = -1;
        if (i < cnt) {
            pay = epay[e0 + i];
            kind = (int)((pay >> 27) & 3u);
        }
        const unsigned mv = __ballot_sync(0xffffffffu, kind == KIND_V);
        const unsigned me = __ballot_sync(0xffffffffu, kind == KIND_E);
        const unsigned mt = __ballot_sync(0xffffffffu, kind == KIND_T);
        if (kind >= 0) {
            const int d = kind == KIND_V ? cv_ + __popc(mv & below)
                                         : (kind == KIND_E ? ce + __popc(me & below) : ct + __popc(mt & below));
            const unsigned long long q = equ[e0 + i];
            R.key[d] = ekey[e0 + i];
            R.qlo[d] = (unsigned)q;
            R.qhi[d] = (unsigned)(q >> 32);
            R.pid[d] = (int)(pay & PAY_PRIM);
        }
        cv_ += __popc(mv);
        ce += __popc(me);
        ct += __popc(mt);
    }
    __syncwarp();
    return kc;
}

// owner test, both-kinematic test and quantized boxes (of one cell when the
// keys agree, which the full tests check)
__device__ __forceinline__ bool prefilter(unsigned la, unsigned ha, unsigned lb, unsigned hb) {
    const unsigned meet = (hb - la) & (ha - lb) & Q_GUARD;
    return ((la | lb) & Q_OWNER) == Q_OWNER && (la & lb & Q_FIXED) == 0 && meet == Q_GUARD;
}

struct RowsOut {
    int *cnt_v, *slots_vt, *cnt_e, *slots_ee;
    int w_vt, w_ee;
    int *overflow;
};

__device__ __forceinline__ void emit(int *cnt, int *slots, int width, int p, int q, int *overflow) {
    const int slot = atomicAdd(&cnt[p], 1);
    if (slot < width) slots[(size_t)p * width + slot] = q;
    else if (slot == width) atomicOr(overflow, OVF_SLOTS);
}

// What the full tests read from device memory.
struct CellData {
    CollView cv;
    const float4 *x0, *x1, *tlo, *thi, *elo, *ehi;
    float dhat;
};

// (vertex entry i of A, triangle entry j of B) past the prefilter
__device__ __forceinline__ void full_vt(const CellRegion &A, int i, const CellRegion &B, int j, const CellData &g,
                                        const RowsOut &o) {
    if (A.key[i] != B.key[j]) return;
    const int v = A.pid[i], t = B.pid[j];
    const int4 T = g.cv.tri[t];
    if (T.x == v || T.y == v || T.z == v) return;
    float3 lo, hi;
    vbox(g.x0, g.x1, v, lo, hi);
    if (!box_overlap(lo, hi, f3(g.tlo[t]), f3(g.thi[t]), g.dhat)) return;
    emit(o.cnt_v, o.slots_vt, o.w_vt, v, t, o.overflow);
}

// (edge entry i of A, edge entry j of B) past the prefilter
__device__ __forceinline__ void full_ee(const CellRegion &A, int i, const CellRegion &B, int j, const CellData &g,
                                        const RowsOut &o) {
    if (A.key[i] != B.key[j]) return;
    int e = A.pid[i], f = B.pid[j];
    const int2 a = g.cv.edge[e], b = g.cv.edge[f];
    if (a.x == b.x || a.x == b.y || a.y == b.x || a.y == b.y) return;
    if (!box_overlap(f3(g.elo[e]), f3(g.ehi[e]), f3(g.elo[f]), f3(g.ehi[f]), g.dhat)) return;
    if (e > f) {
        const int t = e;
        e = f;
        f = t;
    }
    emit(o.cnt_e, o.slots_ee, o.w_ee, e, f, o.overflow);
}

// Survivor queue of one warp: code = i | region_i << 6 | j << 7 | region_j << 13 | ee << 14.
struct PairQueue {
    CellWarp &w;
    const CellData &g;
    const RowsOut &o;
    const unsigned lane;
    int n = 0;  // warp-uniform
    __device__ __forceinline__ void run(unsigned c) const {
        const int i = (int)(c & 63u), j = (int)((c >> 7) & 63u);
        const CellRegion &A = w.r[(c >> 6) & 1u], &B = w.r[(c >> 13) & 1u];
        if (c & (1u << 14)) full_ee(A, i, B, j, g, o);
        else full_vt(A, i, B, j, g, o);
    }
    // every lane calls it (pass: its pair survived the prefilter)
    __device__ __forceinline__ void push(bool pass, unsigned code) {
        const unsigned m = __ballot_sync(0xffffffffu, pass);
        if (pass) w.queue[n + __popc(m & ((1u << lane) - 1u))] = code;
        n += __popc(m);
        if (n >= 32) {  // one survivor per lane
            __syncwarp();
            n -= 32;
            run(w.queue[n + lane]);
            __syncwarp();
        }
    }
    __device__ __forceinline__ void flush() {
        __syncwarp();
        if ((int)lane < n) run(w.queue[lane]);
        n = 0;
        __syncwarp();
    }
};

// every (vertex of region a, triangle of region b): lanes own the triangles
// (their quantized boxes in registers) and run through the vertices
__device__ __forceinline__ void pairs_vt(PairQueue &q, int ra, KindCounts ka, int rb, KindCounts kb) {
    if (ka.v == 0 || kb.t == 0) return;
    const CellRegion &A = q.w.r[ra], &B = q.w.r[rb];
    const int t0 = kb.v + kb.e;
    for (int tb = 0; tb < kb.t; tb += 32) {  // warp-uniform
        const bool own = tb + (int)q.lane < kb.t;
        const int j = t0 + (own ? tb + (int)q.lane : 0);
        const unsigned lb = B.qlo[j], hb = B.qhi[j];
        for (int i = 0; i < ka.v; ++i) {
            const bool pass = own && prefilter(A.qlo[i], A.qhi[i], lb, hb);
            q.push(pass, (unsigned)i | ((unsigned)ra << 6) | ((unsigned)j << 7) | ((unsigned)rb << 13));
        }
    }
}

// every unordered pair of edges of region a: lane entry ii meets ii + d
// (mod n) for d = 1 .. (n - 1) / 2, and, for even n, ii + n / 2 when ii < n / 2
__device__ __forceinline__ void pairs_ee_within(PairQueue &q, int ra, KindCounts ka) {
    const int n = ka.e;
    if (n < 2) return;
    const CellRegion &A = q.w.r[ra];
    const int e0 = ka.v, h = (n - 1) / 2, dlim = h + ((n & 1) == 0 ? 1 : 0);
    for (int ib = 0; ib < n; ib += 32) {  // warp-uniform
        const int ii = ib + (int)q.lane;
        const bool own = ii < n;
        const int i = e0 + (own ? ii : 0);
        const unsigned la = A.qlo[i], ha = A.qhi[i];
        const int dmax = own ? h + (((n & 1) == 0 && ii < n / 2) ? 1 : 0) : 0;
        int jj = own ? ii : 0;
        for (int d = 1; d <= dlim; ++d) {
            if (++jj >= n) jj -= n;
            const int j = e0 + jj;
            const bool pass = d <= dmax && prefilter(la, ha, A.qlo[j], A.qhi[j]);
            q.push(pass, (unsigned)i | ((unsigned)ra << 6) | ((unsigned)j << 7) | ((unsigned)ra << 13) | (1u << 14));
        }
    }
}

// every (edge of region a, edge of region b), two chunks of one bucket
__device__ __forceinline__ void pairs_ee_across(PairQueue &q, int ra, KindCounts ka, int rb, KindCounts kb) {
    if (ka.e == 0 || kb.e == 0) return;
    const CellRegion &A = q.w.r[ra], &B = q.w.r[rb];
    for (int ib = 0; ib < ka.e; ib += 32) {  // warp-uniform
        const bool own = ib + (int)q.lane < ka.e;
        const int i = ka.v + (own ? ib + (int)q.lane : 0);
        const unsigned la = A.qlo[i], ha = A.qhi[i];
        for (int jj = 0; jj < kb.e; ++jj) {
            const int j = kb.v + jj;
            const bool pass = own && prefilter(la, ha, B.qlo[j], B.qhi[j]);
            q.push(pass, (unsigned)i | ((unsigned)ra << 6) | ((unsigned)j << 7) | ((unsigned)rb << 13) | (1u << 14));
        }
    }
}

template <int W>
__global__ void __launch_bounds__(W * 32) k_cell_pairs(CellData g, int T, const int *__restrict__ bcnt,
                                                       const int *__restrict__ bstart,
                                                       const unsigned long long *__restrict__ ekey,
                                                       const unsigned int *__restrict__ epay,
                                                       const unsigned long long *__restrict__ equ, RowsOut o,
                                                       int *work, const long long *hash_total, long long cap_ent) {
    extern __shared__ __align__(16) unsigned char cell_smem[];  // W CellWarp
    if (*hash_total > cap_ent) return;  // table not filled: no candidates (the pass is redone)
    const unsigned lane = threadIdx.x & 31;
    CellWarp &cw = reinterpret_cast<CellWarp *>(cell_smem)[threadIdx.x >> 5];
    PairQueue q{cw, g, o, lane};
    for (;;) {
        int b0 = 0;
        if (lane == 0) b0 = atomicAdd(work, 32);
        b0 = __shfl_sync(0xffffffffu, b0, 0);
        if (b0 >= T) break;
        const int b = b0 + (int)lane;
        const int m = b < T ? bcnt[b] : 0;
        const int st = b < T ? bstart[b] : 0;
        unsigned todo = __ballot_sync(0xffffffffu, m >= 2);
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int mb = __shfl_sync(0xffffffffu, m, l);
            const int eb = __shfl_sync(0xffffffffu, st, l);
            const int nch = (mb + CELL_CHUNK - 1) / CELL_CHUNK;
            for (int ca = 0; ca < nch; ++ca) {
                const KindCounts a = load_chunk(cw.r[0], ekey, epay, equ, eb + ca * CELL_CHUNK,
                                                min(CELL_CHUNK, mb - ca * CELL_CHUNK), lane);
                pairs_vt(q, 0, a, 0, a);
                pairs_ee_within(q, 0, a);
                for (int cb = ca + 1; cb < nch; ++cb) {
                    const KindCounts c = load_chunk(cw.r[1], ekey, epay, equ, eb + cb * CELL_CHUNK,
                                                    min(CELL_CHUNK, mb - cb * CELL_CHUNK), lane);
                    pairs_vt(q, 0, a, 1, c);
                    pairs_vt(q, 1, c, 0, a);
                    pairs_ee_across(q, 0, a, 1, c);
                    q.flush();  // region 1 is reloaded next
                }
                q.flush();  // region 0 is reloaded next
            }
        }
    }
}

// out[off[p] + k] = (p, k-th smallest of row p) for k < cnt[p]: the list
// comes out sorted by (primary, secondary) whatever order the appends took.
// A warp takes 32 rows; for each non-empty one its lanes hold the row's
// entries and place each at its rank (entries of a row are distinct).
__global__ void k_compact_rows(int np, const int *__restrict__ cnt, const int *__restrict__ off,
                               const int *__restrict__ slots, int width, const long long *total, long long cap,
                               int2 *__restrict__ out) {
    const unsigned lane = threadIdx.x & 31;
    const int p0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31;
    if (p0 >= np || *total > cap) return;  // uniform per warp
    const int p = p0 + (int)lane;
    const int c = p < np ? min(cnt[p], width) : 0;
    const int o = p < np ? off[p] : 0;
    unsigned todo = __ballot_sync(0xffffffffu, c > 0);
    while (todo) {
        const int l = __ffs(todo) - 1;
        todo &= todo - 1u;
        const int q = p0 + l;
        const int cq = __shfl_sync(0xffffffffu, c, l), oq = __shfl_sync(0xffffffffu, o, l);
        const int *row = slots + (size_t)q * width;
        for (int k0 = 0; k0 < cq; k0 += 32) {  // entries k0 + lane ranked against the whole row
            const int k = k0 + (int)lane;
            const int v = k < cq ? row[k] : 0x7fffffff;
            int rank = 0;
            for (int j0 = 0; j0 < cq; j0 += 32) {
                const int w = j0 + (int)lane < cq ? row[j0 + lane] : 0x7fffffff;
                const int nj = min(32, cq - j0);
                for (int j = 0; j < nj; ++j) rank += __shfl_sync(0xffffffffu, w, j) < v ? 1 : 0;
            }
            if (k < cq) out[oq + rank] = make_int2(q, v);
        }
    }
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
    if ((long long)cv.nv + cv.ne + cv.nt >= (1LL << 27))
        throw Error(PDC_ERR_ARG, "broad phase: 2^27 or more vertices, edges and triangles");
    // about one bucket per primitive: occupied cells are far fewer, so most
    // buckets hold a single cell
    T = (int)pow2((long long)cv.nv + cv.ne + cv.nt + 1024);
    bcnt.alloc(T);
    bstart.alloc(T);
    bfill.alloc(T);
    work.alloc(1);
    cap_ent = cap_ent_;
    ekey.alloc(cap_ent);
    epay.alloc(cap_ent);
    equ.alloc(cap_ent);
    tlo.alloc(cv.nt);
    thi.alloc(cv.nt);
    elo.alloc(cv.ne);
    ehi.alloc(cv.ne);
    cnt_v.alloc(cv.nv);
    for (int k = 0; k < 2; ++k) {
        off_v[k].alloc(std::max(cv.nv, 1));
        off_e[k].alloc(std::max(cv.ne, 1));
        off_ok[k] = false;
    }
    cnt_e.alloc(cv.ne);
    slots_vt.alloc((size_t)cv.nv * w_vt);
    slots_ee.alloc((size_t)cv.ne * w_ee);
    long long mx = std::max<long long>(T, std::max<long long>(cv.nv, cv.ne));
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
        ekey.alloc(cap_ent);
        epay.alloc(cap_ent);
        equ.alloc(cap_ent);
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
    hash_pass(s, cv, x0, x1, dhat, overflow, vt[nw], ee[nw], cnt_vt_d[nw], cnt_ee_d[nw], nw);
    off_ok[nw] = true;
    cur = nw;
    sup_ok = false;
    k_pccd_force<<<1, 1, 0, s>>>(pccd);  // new lists: the next partial-CCD pass scans them all
    PDC_LAUNCH_CK();
}

void BroadPhase::hash_pass(cudaStream_t s, const CollView &cv, const float4 *x0, const float4 *x1, float dhat,
                           int *overflow, int2 *out_vt, int2 *out_ee, long long *out_nvt, long long *out_nee,
                           int slot) {
    long long *tot = totals.p;
    const int np = cv.nv + cv.ne + cv.nt;
    const unsigned mask = (unsigned)(T - 1);
    CellData g;
    g.cv = cv;
    g.x0 = x0;
    g.x1 = x1;
    g.tlo = tlo;
    g.thi = thi;
    g.elo = elo;
    g.ehi = ehi;
    g.dhat = dhat;
    RowsOut o;
    o.cnt_v = cnt_v;
    o.slots_vt = slots_vt;
    o.cnt_e = cnt_e;
    o.slots_ee = slots_ee;
    o.w_vt = w_vt;
    o.w_ee = w_ee;
    o.overflow = overflow;
    // boxes, grid (cell = mean triangle extent x scale), cell table, the VT
    // and EE pairs of every cell into the per-primary rows (w warps a block)
    auto build = [&](float scale, int w) {
        PDC_CK(cudaMemsetAsync(gp.p, 0, sizeof(GridParams), s));
        BP_PROF("bp_boxes", if (cv.nt) k_tri_boxes<<<nblk(cv.nt, 256), 256, 0, s>>>(cv, x0, x1, tlo, thi, gp);
                if (cv.ne) k_edge_boxes<<<nblk(cv.ne, 256), 256, 0, s>>>(cv, x0, x1, elo, ehi);
                k_grid_params<<<1, 1, 0, s>>>(gp, cv.nt, dhat, scale));
        PDC_LAUNCH_CK();
        // ---- cell table: count per bucket, prefix sum, fill
        BP_PROF("bp_hash_build", bcnt.zero(s); bfill.zero(s);
        if (np) {
            k_cell_insert<<<nblk(np, 256), 256, 0, s>>>(cv, x0, x1, tlo, thi, elo, ehi, gp, dhat, mask, bcnt, bstart,
                                                        bfill, ekey, epay, equ, 0, tot, cap_ent, overflow);
            PDC_LAUNCH_CK();
        }
        exclusive_scan(s, bcnt, bstart, T, scratch, tot);
        k_check_cap<<<1, 1, 0, s>>>(tot, cap_ent, OVF_HASH, overflow, tot + 4);
        if (np) {
            k_cell_insert<<<nblk(np, 256), 256, 0, s>>>(cv, x0, x1, tlo, thi, elo, ehi, gp, dhat, mask, bcnt, bstart,
                                                        bfill, ekey, epay, equ, 1, tot, cap_ent, overflow);
            PDC_LAUNCH_CK();
        });
        if (prof) prof->begin(s, "bp_cell_pairs", 0.0);
        cnt_v.zero(s);
        cnt_e.zero(s);
        work.zero(s);
        if (np) {
            // 64 resident warps an SM for each shape (2.8 KB of shared memory a warp)
#define PDC_CELLS(W, B)                                                                                              \
    do {                                                                                                             \
        const int smem = (W) * (int)sizeof(CellWarp);                                                               \
        static bool attr = false;                                                                                    \
        if (!attr) {                                                                                                 \
            PDC_CK(cudaFuncSetAttribute(k_cell_pairs<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));        \
            attr = true;                                                                                             \
        }                                                                                                            \
        k_cell_pairs<W><<<152 * (B), (W) * 32, smem, s>>>(g, T, bcnt, bstart, ekey, epay, equ, o, work, tot,      \
                                                          cap_ent);                                                  \
    } while (0)
            if (w == 4) PDC_CELLS(4, 16);
            else if (w == 16) PDC_CELLS(16, 4);
            else PDC_CELLS(8, 8);
#undef PDC_CELLS
            PDC_LAUNCH_CK();
        }
        if (prof) prof->end(s);
    };
    // tuned on the TUNE_PASS-th pass after the request: the first passes of a
    // run see the cloth nearly at rest, smaller boxes than later on
    constexpr int TUNE_PASS = 8;
    if (tune_cells && ++tune_wait >= TUNE_PASS) {
        // every candidate finds the same pairs (the rows differ only in order,
        // which the compaction sorts out): time each whole build, keep the
        // fastest grid, then the fastest block shape on it
        tune_cells = false;
        tune_wait = 0;
        const float grids[3] = {1.f, 1.5f, 2.f};
        const int warps[3] = {4, 8, 16};
        cudaEvent_t e[4];
        for (auto &ev : e) PDC_CK(cudaEventCreate(&ev));
        auto sweep = [&](float *ms, auto &&run) {
            PDC_CK(cudaEventRecord(e[0], s));
            for (int k = 0; k < 3; ++k) {
                run(k);
                PDC_CK(cudaEventRecord(e[k + 1], s));
            }
            PDC_CK(cudaEventSynchronize(e[3]));
            for (int k = 0; k < 3; ++k) PDC_CK(cudaEventElapsedTime(&ms[k], e[k], e[k + 1]));
            int best = 0;  // the fastest, once all are timed
            for (int k = 1; k < 3; ++k)
                if (ms[k] < ms[best]) best = k;
            return best;
        };
        build(cell_scale * cell_grid, cell_warps);  // warm-up
        cell_grid = grids[sweep(grid_ms, [&](int k) { build(cell_scale * grids[k], cell_warps); })];
        cell_warps = warps[sweep(cell_ms, [&](int k) { build(cell_scale * cell_grid, warps[k]); })];
        for (auto &ev : e) cudaEventDestroy(ev);
    } else {
        build(cell_scale * cell_grid, cell_warps);
    }
    // ---- rows -> sorted pair lists
    if (prof) prof->begin(s, "bp_compact", 0.0);
    int *ov = off_v[slot], *oe = off_e[slot];
    exclusive_scan(s, cnt_v, ov, cv.nv, scratch, tot + 2);
    k_check_cap<<<1, 1, 0, s>>>(tot + 2, cap_vt, OVF_VT, overflow, out_nvt);
    if (cv.nv) {
        k_compact_rows<<<nblk(cv.nv, 256), 256, 0, s>>>(cv.nv, cnt_v, ov, slots_vt, w_vt, tot + 2, cap_vt, out_vt);
        PDC_LAUNCH_CK();
    }
    exclusive_scan(s, cnt_e, oe, cv.ne, scratch, tot + 3);
    k_check_cap<<<1, 1, 0, s>>>(tot + 3, cap_ee, OVF_EE, overflow, out_nee);
    if (cv.ne) {
        k_compact_rows<<<nblk(cv.ne, 256), 256, 0, s>>>(cv.ne, cnt_e, oe, slots_ee, w_ee, tot + 3, cap_ee, out_ee);
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
    hash_pass(s, cv, x0, x1, gap, overflow, sup_vt, sup_ee, sup_cnt.p, sup_cnt.p + 1, cur ^ 1);
    off_ok[cur ^ 1] = false;  // those offsets are the superset's
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
    off_ok[nw] = false;  // a filtered list has no segment offsets
    cur = nw;
    k_pccd_force<<<1, 1, 0, s>>>(pccd);  // new lists: the next partial-CCD pass scans them all
    PDC_LAUNCH_CK();
}

}  // namespace pdc
