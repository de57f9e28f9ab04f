// k_remesh.cu -- adaptation of a single-mesh context on the device (Sec. 2.4
// and the adaptive runs of Sec. 3): the refine/coarsen plan with its 2:1
// balance (reading R28), the families of the solution transfer, and the
// mesh tables of the adapted quadtree (face kinds and neighbours, mortars,
// mortar nodes and the blocks of the mortar limiting kernel), written into
// device buffers. Every table equals the one the host builder forms for the
// same leaves (idp_host.cu: build_mesh, host_mortar_tables, idp_amr_plan).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "idp_remesh.h"

namespace idp {
namespace rm {

enum : int { FT_CONF_ = 0, FT_BND_ = 1, FT_MLARGE_ = 2, FT_MSLO_ = 3, FT_MSHI_ = 4 };
enum : int { ERR_DUP = 1, ERR_BALANCE = 2, ERR_PENDING = 4, ERR_NODE3 = 8, ERR_FOREIGN = 16 };

__device__ __forceinline__ unsigned long long leaf_key(int l, long long x, long long y) {
    return ((unsigned long long)l << 58) | ((unsigned long long)x << 29) | (unsigned long long)y;
}
__device__ __forceinline__ unsigned long long mix(unsigned long long k) {
    k ^= k >> 33; k *= 0xff51afd7ed558ccdull; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ull; k ^= k >> 33;
    return k;
}
constexpr unsigned long long EMPTY = ~0ull;

__device__ __forceinline__ int side_of(const int4 &v, int s) { return s == 0 ? v.x : (s == 1 ? v.y : (s == 2 ? v.z : v.w)); }
__device__ __forceinline__ int side_of(const uchar4 &v, int s) { return s == 0 ? v.x : (s == 1 ? v.y : (s == 2 ? v.z : v.w)); }
__device__ __forceinline__ void set_side(int4 &v, int s, int x) { if (s == 0) v.x = x; else if (s == 1) v.y = x; else if (s == 2) v.z = x; else v.w = x; }
__device__ __forceinline__ void set_side(uchar4 &v, int s, int x) {
    const unsigned char c = (unsigned char)x;
    if (s == 0) v.x = c; else if (s == 1) v.y = c; else if (s == 2) v.z = c; else v.w = c;
}

// ---------------------------------------------------------------- scans ----
// exclusive scan of n ints in blocks of 1024 (warp scans), block totals out
__global__ void __launch_bounds__(1024) k_scan_block(const int *in, int *out, int *bsum, int n) {
    __shared__ int ws[32];
    const int i = blockIdx.x * 1024 + threadIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = i < n ? in[i] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    const int pre = (w > 0 ? ws[w - 1] : 0) + x - v;
    if (i < n) out[i] = pre;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = ws[31];
}

__global__ void k_scan_add(int *out, const int *boff, int n) {
    const int i = blockIdx.x * 1024 + threadIdx.x;
    if (i < n && blockIdx.x > 0) out[i] += boff[blockIdx.x];
}

// out = exclusive scan of in (n entries), total in out[n]; tmp: scan_tmp_ints(n)
void exclusive_scan(const int *in, int *out, int n, int *tmp, cudaStream_t st) {
    const int nb = (n + 1023) / 1024;
    int *bsum = tmp, *boff = tmp + nb + 1;
    k_scan_block<<<std::max(nb, 1), 1024, 0, st>>>(in, out, bsum, n);
    if (nb > 1) {
        exclusive_scan(bsum, boff, nb, tmp + 2 * (nb + 1), st);
        k_scan_add<<<nb, 1024, 0, st>>>(out, boff, n);
        // total = last block's offset + its sum
        cudaMemcpyAsync(out + n, boff + nb, sizeof(int), cudaMemcpyDeviceToDevice, st);
    } else {
        cudaMemcpyAsync(out + n, bsum, sizeof(int), cudaMemcpyDeviceToDevice, st);
    }
}

size_t scan_tmp_ints(int n) {
    size_t t = 0;
    for (int m = n; m > 1;) { const int nb = (m + 1023) / 1024; t += 2 * (size_t)(nb + 1); m = nb; }
    return t + 8;
}

// ----------------------------------------------------------------- plan ----
__global__ void k_marks(const double *ind, const int8_t *lev, int K, double rt, double ct, int minl, int maxl,
                        int *mark) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
        int m = 0;
        if (ind[e] > rt && lev[e] < maxl) m = 1;
        else if (ind[e] < ct && lev[e] > minl) m = -1;
        mark[e] = m;
    }
}

// The four siblings of leaf e, children c = cx + 2 cy of its parent, found
// across conforming faces inside the parent (a sibling that is not a leaf of
// e's level leaves the family incomplete: -1).
__device__ void family(const int4 *fnbr, const uchar4 *ftype, const int *ix, const int *iy, int e, int f[4]) {
    const int cx = ix[e] & 1, cy = iy[e] & 1;
    for (int c = 0; c < 4; ++c) f[c] = -1;
    f[cx + 2 * cy] = e;
    const int sx = cx == 0 ? 1 : 0, sy = cy == 0 ? 3 : 2;   // sides toward the x and y siblings
    const int ex = side_of(ftype[e], sx) == FT_CONF_ ? side_of(fnbr[e], sx) : -1;
    const int ey = side_of(ftype[e], sy) == FT_CONF_ ? side_of(fnbr[e], sy) : -1;
    f[(cx ^ 1) + 2 * cy] = ex;
    f[cx + 2 * (cy ^ 1)] = ey;
    int exy = -1;
    if (ex >= 0 && side_of(ftype[ex], sy) == FT_CONF_) exy = side_of(fnbr[ex], sy);
    else if (ey >= 0 && side_of(ftype[ey], sx) == FT_CONF_) exy = side_of(fnbr[ey], sx);
    f[(cx ^ 1) + 2 * (cy ^ 1)] = exy;
}

// a family coarsens only when all four siblings are leaves marked -1
__global__ void k_family(const int4 *fnbr, const uchar4 *ftype, const int *ix, const int *iy, int K,
                         const int *mark_in, int *mark_out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
        int m = mark_in[e];
        if (m == -1) {
            int f[4];
            family(fnbr, ftype, ix, iy, e, f);
            bool ok = true;
            for (int c = 0; c < 4; ++c) ok = ok && f[c] >= 0 && mark_in[f[c]] == -1;
            if (!ok) m = 0;
        }
        mark_out[e] = m;
    }
}

// One sweep of the 2:1 balance: a neighbour whose target level exceeds e's by
// two or more refines e, or, if e was to coarsen, keeps e's family. Marks only
// rise (-1 -> 0 -> 1), so the sweeps reach the host loop's fixed point.
__global__ void k_balance(const int4 *fnbr, const uchar4 *ftype, const int32_t *m_large, const int2 *m_small,
                          const int8_t *lev, const int *ix, const int *iy, int K, int *mark, int *changed) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
        const int me = mark[e];
        const int fe = lev[e] + me;
        bool up = false;
        for (int s = 0; s < 4 && !up; ++s) {
            const int ft = side_of(ftype[e], s), nb = side_of(fnbr[e], s);
            int n[2] = {-1, -1};
            if (ft == FT_CONF_) n[0] = nb;
            else if (ft == FT_MLARGE_) { n[0] = m_small[nb].x; n[1] = m_small[nb].y; }
            else if (ft == FT_MSLO_ || ft == FT_MSHI_) n[0] = m_large[nb];
            for (int t = 0; t < 2; ++t)
                if (n[t] >= 0 && lev[n[t]] + mark[n[t]] - fe >= 2) up = true;
        }
        if (!up) continue;
        if (me == -1) {
            int f[4];
            family(fnbr, ftype, ix, iy, e, f);
            for (int c = 0; c < 4; ++c)
                if (f[c] >= 0 && atomicMax(&mark[f[c]], 0) < 0) *changed = 1;
        } else if (me == 0) {
            atomicMax(&mark[e], 1);
            *changed = 1;
        }
    }
}

// new leaves per old element: 4 (refined), 1 (kept, or the first leaf of a
// coarsened family), 0 (the other three); transfer families: 1 per refined
// element and per coarsened family
__global__ void k_emit_count(const int4 *fnbr, const uchar4 *ftype, const int *ix, const int *iy, int K,
                             const int *mark, int *cnt, int *fcnt) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
        const int m = mark[e];
        int c = 1, fc = 0;
        if (m == 1) { c = 4; fc = 1; }
        else if (m == -1) {
            int f[4];
            family(fnbr, ftype, ix, iy, e, f);
            const int mn = min(min(f[0], f[1]), min(f[2], f[3]));
            c = mn == e ? 1 : 0;
            fc = c;
        }
        cnt[e] = c;
        fcnt[e] = fc;
    }
}

__global__ void k_emit(const int4 *fnbr, const uchar4 *ftype, const int8_t *lev, const int *ix, const int *iy,
                       int K, const int *mark, const int *off, const int *foff, int8_t *nlev, int *nix, int *niy,
                       int *kind, int4 *src, int4 *fam) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
        const int m = mark[e], o = off[e], l = lev[e];
        const long long x = ix[e], y = iy[e];
        if (m == 1) {
            for (int c = 0; c < 4; ++c) {
                nlev[o + c] = (int8_t)(l + 1);
                nix[o + c] = (int)(2 * x + (c & 1));
                niy[o + c] = (int)(2 * y + (c >> 1));
                kind[o + c] = 1;
                src[o + c] = make_int4(e, c, -1, -1);
            }
            fam[foff[e]] = make_int4(o, 4, 0, e);
        } else if (m == -1) {
            int f[4];
            family(fnbr, ftype, ix, iy, e, f);
            if (min(min(f[0], f[1]), min(f[2], f[3])) != e) continue;
            nlev[o] = (int8_t)(l - 1);
            nix[o] = (int)(x >> 1);
            niy[o] = (int)(y >> 1);
            kind[o] = 2;
            src[o] = make_int4(f[0], f[1], f[2], f[3]);
            fam[foff[e]] = make_int4(o, 1, 1, o);
        } else {
            nlev[o] = (int8_t)l;
            nix[o] = (int)x;
            niy[o] = (int)y;
            kind[o] = 0;
            src[o] = make_int4(e, -1, -1, -1);
        }
    }
}

// ------------------------------------------------------------ the mesh ----
__global__ void k_hash_clear(unsigned long long *keys, int cap) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cap; k += gridDim.x * blockDim.x) keys[k] = EMPTY;
}

__global__ void k_hash_insert(const int8_t *lev, const int *ix, const int *iy, int K, unsigned long long *keys,
                              int *vals, int mask, int *err) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
        const unsigned long long key = leaf_key(lev[e], ix[e], iy[e]);
        unsigned long long h = mix(key) & (unsigned long long)mask;
        for (int probe = 0; probe <= mask; ++probe) {
            const unsigned long long prev = atomicCAS(&keys[h], EMPTY, key);
            if (prev == EMPTY) { vals[h] = e; break; }
            if (prev == key) { atomicOr(err, ERR_DUP); break; }
            h = (h + 1) & (unsigned long long)mask;
        }
    }
}

__device__ __forceinline__ int hash_find(const unsigned long long *keys, const int *vals, int mask, int l, long long x,
                                         long long y) {
    if (l < 0) return -1;
    const unsigned long long key = leaf_key(l, x, y);
    unsigned long long h = mix(key) & (unsigned long long)mask;
    for (int probe = 0; probe <= mask; ++probe) {
        const unsigned long long k = keys[h];
        if (k == key) return vals[h];
        if (k == EMPTY) return -1;
        h = (h + 1) & (unsigned long long)mask;
    }
    return -1;
}

// geometry, derived constants and simulation id, as the host forms them
__global__ void k_geom(const RemeshMesh M, const int8_t *lev, const int *ix, const int *iy, int K, Geo *geom,
                       GeoC *geoc, int *sim) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
        const int l = lev[e];
        const double dx = (M.x1 - M.x0) / ((double)M.nx0 * (double)(1LL << l));
        const double dy = (M.y1 - M.y0) / ((double)M.ny0 * (double)(1LL << l));
        Geo g;
        // rounded as the host builder rounds it (no contraction into an FMA)
        g.x = __dadd_rn(M.x0, __dmul_rn((double)ix[e], dx));
        g.y = __dadd_rn(M.y0, __dmul_rn((double)iy[e], dy));
        g.z = dx; g.w = dy;
        geom[e] = g;
        GeoC q;
        q.iA4 = 4.0 / (g.z * g.w); q.A4 = 0.25 * (g.z * g.w);
        q.hx = 0.5 * g.z; q.hy = 0.5 * g.w; q.qx = 0.25 * g.z; q.qy = 0.25 * g.w;
        q.hxf = (float)q.hx; q.hyf = (float)q.hy; q.qxf = (float)q.qx; q.qyf = (float)q.qy; q.A4f = (float)q.A4;
        q.pad = 0.0f;
        geoc[e] = q;
        sim[e] = 0;
    }
}

// per element side: conforming neighbour, boundary, the large side of a
// mortar (flag), or the small side of one (pending until the mortars are set)
__global__ void k_faces(const RemeshMesh M, const int8_t *lev, const int *ix, const int *iy, int K,
                        const unsigned long long *keys, const int *vals, int mask, int4 *fnbr, uchar4 *ftype,
                        int *mflag, int2 *msmall_cand, int *err) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 4 * K; k += gridDim.x * blockDim.x) {
        const int e = k >> 2, s = k & 3, l = lev[e];
        const long long nxl = (long long)M.nx0 << l, nyl = (long long)M.ny0 << l;
        long long qx = ix[e] + (s == 0 ? -1 : (s == 1 ? 1 : 0));
        long long qy = iy[e] + (s == 2 ? -1 : (s == 3 ? 1 : 0));
        const bool outside = qx < 0 || qx >= nxl || qy < 0 || qy >= nyl;
        int kind = FT_BND_, nb = -1, flag = 0;
        int2 cand = make_int2(-1, -1);
        if (!outside || M.bc[s] == 0) {   // periodic
            qx = (qx + nxl) % nxl;
            qy = (qy + nyl) % nyl;
            const int f = hash_find(keys, vals, mask, l, qx, qy);
            if (f >= 0) { kind = FT_CONF_; nb = f; }
            else if (l > 0 && hash_find(keys, vals, mask, l - 1, qx >> 1, qy >> 1) >= 0) { kind = -1; }
            else {
                long long ax, ay, bx, by;
                if (s < 2) { ax = bx = 2 * qx + (s == 0 ? 1 : 0); ay = 2 * qy; by = 2 * qy + 1; }
                else { ay = by = 2 * qy + (s == 2 ? 1 : 0); ax = 2 * qx; bx = 2 * qx + 1; }
                const int a = hash_find(keys, vals, mask, l + 1, ax, ay), b = hash_find(keys, vals, mask, l + 1, bx, by);
                if (a < 0 || b < 0) atomicOr(err, ERR_BALANCE);
                flag = 1;
                cand = make_int2(a, b);
                kind = FT_MLARGE_;
            }
        }
        mflag[k] = flag;
        msmall_cand[k] = cand;
        // small sides (kind -1) are written by the mortars below
        if (kind != -1) {
            reinterpret_cast<int *>(&fnbr[e])[s] = nb;
            reinterpret_cast<unsigned char *>(&ftype[e])[s] = (unsigned char)(kind == FT_MLARGE_ ? FT_MLARGE_ : kind);
        } else {
            reinterpret_cast<int *>(&fnbr[e])[s] = -1;
            reinterpret_cast<unsigned char *>(&ftype[e])[s] = 255;   // pending
        }
    }
}

// the mortars in element-major, side order (the host builder's order)
__global__ void k_mortars(const int *mflag, const int *moff, const int2 *cand, int K, int4 *fnbr, uchar4 *ftype,
                          int32_t *m_large, int2 *m_small, int32_t *m_info) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 4 * K; k += gridDim.x * blockDim.x) {
        if (!mflag[k]) continue;
        const int e = k >> 2, s = k & 3, m = moff[k];
        const int low = (s == 1 || s == 3) ? 1 : 0;
        m_large[m] = e;
        m_small[m] = cand[k];
        m_info[m] = (s >> 1) | (low << 1);
        reinterpret_cast<int *>(&fnbr[e])[s] = m;
        const int dir = s >> 1;
        const int s_small = dir == 0 ? (low ? 0 : 1) : (low ? 2 : 3);
        const int a = cand[k].x, b = cand[k].y;
        if (a >= 0) {
            reinterpret_cast<int *>(&fnbr[a])[s_small] = m;
            reinterpret_cast<unsigned char *>(&ftype[a])[s_small] = (unsigned char)FT_MSLO_;
        }
        if (b >= 0) {
            reinterpret_cast<int *>(&fnbr[b])[s_small] = m;
            reinterpret_cast<unsigned char *>(&ftype[b])[s_small] = (unsigned char)FT_MSHI_;
        }
    }
}

__global__ void k_check_pending(const uchar4 *ftype, int K, int *err) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 4 * K; k += gridDim.x * blockDim.x)
        if (reinterpret_cast<const unsigned char *>(ftype)[k] == 255) atomicOr(err, ERR_PENDING);
}

__device__ __forceinline__ long long slot_node(int NP, int m, int q, const int32_t *m_large, const int2 *m_small,
                                               const int32_t *m_info) {
    const int NN = NP * NP, dir = m_info[m] & 1, low = (m_info[m] >> 1) & 1;
    const int sL = dir == 0 ? (low ? 1 : 0) : (low ? 3 : 2), sS = sL ^ 1;
    int e, s, t;
    if (q < NP) { e = m_large[m]; s = sL; t = q; }
    else { e = ((q - NP) / NP == 0) ? m_small[m].x : m_small[m].y; s = sS; t = (q - NP) % NP; }
    const int i = s == 0 ? 0 : (s == 1 ? NP - 1 : t), j = s == 2 ? 0 : (s == 3 ? NP - 1 : t);
    return (long long)e * NN + j * NP + i;
}

__global__ void k_node_fill(int *a, long long n, int v) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) a[k] = v;
}

// first (smallest) slot of every mortar node
__global__ void k_node_first(int NP, int M, const int32_t *m_large, const int2 *m_small, const int32_t *m_info,
                             int *first) {
    const int Q = 3 * NP;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M * Q; k += gridDim.x * blockDim.x)
        atomicMin(&first[slot_node(NP, k / Q, k % Q, m_large, m_small, m_info)], k);
}

// second slot; a third is an invalid mesh
__global__ void k_node_second(int NP, int M, const int32_t *m_large, const int2 *m_small, const int32_t *m_info,
                              const int *first, int *second, int *third) {
    const int Q = 3 * NP;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M * Q; k += gridDim.x * blockDim.x) {
        const long long g = slot_node(NP, k / Q, k % Q, m_large, m_small, m_info);
        if (first[g] != k) atomicMin(&second[g], k);
    }
    (void)third;
}

__global__ void k_node_third(int NP, int M, const int32_t *m_large, const int2 *m_small, const int32_t *m_info,
                             const int *first, const int *second, int *err) {
    const int Q = 3 * NP;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M * Q; k += gridDim.x * blockDim.x) {
        const long long g = slot_node(NP, k / Q, k % Q, m_large, m_small, m_info);
        if (first[g] != k && second[g] != k) atomicOr(err, ERR_NODE3);
    }
}

// Slots of one block of the mortar limiting kernel: W mortars of Q slots,
// at most 114 for every degree (W Q <= 19 x 6), so the foreign candidates of
// a block (at most one per slot) fit one warp's list.
constexpr int FCAP = 128;
constexpr int MB_WARPS = 4;   // blocks of the limiting kernel per CTA, one warp each

// One warp per block b of the mortar limiting kernel: its owned nodes (the
// nodes whose first slot is in the block) in slot order with their two
// slots, and its foreign mortars (the mortars of the second slots outside
// the block) ascending and unique. With null outputs only the counts.
__device__ void warp_block(int NP, int W, int M, int b, const int32_t *m_large, const int2 *m_small,
                           const int32_t *m_info, const int *first, const int *second, int *cand, int *keep,
                           int32_t *node_out, int2 *slot_out, int32_t *fore_out, int *n_out, int *nf_out, int *err) {
    const int lane = threadIdx.x & 31, Q = 3 * NP;
    const int s0 = b * W * Q, s1 = min(M, b * W + W) * Q;
    if (s1 - s0 > FCAP) {
        if (lane == 0) { atomicOr(err, ERR_FOREIGN); *n_out = 0; *nf_out = 0; }
        return;
    }
    const unsigned lt = (1u << lane) - 1u;
    int n = 0, nc = 0;
    for (int base = s0; base < s1; base += 32) {
        const int sl = base + lane;
        bool own = false;
        int s2 = -1, fm = -1;
        long long g = 0;
        if (sl < s1) {
            g = slot_node(NP, sl / Q, sl % Q, m_large, m_small, m_info);
            own = first[g] == sl;
            if (own) {
                s2 = second[g] == 0x7fffffff ? -1 : second[g];
                if (s2 >= 0 && (s2 / Q) / W != b) fm = s2 / Q;
            }
        }
        const unsigned bo = __ballot_sync(0xffffffffu, own), bf = __ballot_sync(0xffffffffu, fm >= 0);
        if (own && node_out) {
            const int q = n + __popc(bo & lt);
            node_out[q] = (int32_t)g;
            slot_out[q] = make_int2(sl, s2);
        }
        if (fm >= 0) cand[nc + __popc(bf & lt)] = fm;
        n += __popc(bo);
        nc += __popc(bf);
    }
    __syncwarp();
    // the first occurrence of each candidate value is kept; its place is the
    // number of kept values below it
    for (int i = lane; i < nc; i += 32) {
        int k = 1;
        for (int j = 0; j < i && k; ++j) k = cand[j] != cand[i];
        keep[i] = k;
    }
    __syncwarp();
    int nf = 0;
    for (int i = lane; i < nc; i += 32) {
        nf += keep[i];
        if (fore_out && keep[i]) {
            int pos = 0;
            for (int j = 0; j < nc; ++j) pos += keep[j] && cand[j] < cand[i];
            fore_out[pos] = cand[i];
        }
    }
    for (int o = 16; o > 0; o >>= 1) nf += __shfl_xor_sync(0xffffffffu, nf, o);
    __syncwarp();
    if (lane == 0) { *n_out = n; *nf_out = nf; }
}

__global__ void __launch_bounds__(32 * MB_WARPS) k_mb_count(int NP, int W, int M, int nb, const int32_t *m_large,
                                                           const int2 *m_small, const int32_t *m_info,
                                                           const int *first, const int *second, int *ncnt, int *fcnt,
                                                           int *fmax, int *err) {
    __shared__ int cand[MB_WARPS][FCAP], keep[MB_WARPS][FCAP];
    const int w = threadIdx.x >> 5, b = blockIdx.x * MB_WARPS + w;
    if (b >= nb) return;
    warp_block(NP, W, M, b, m_large, m_small, m_info, first, second, cand[w], keep[w], nullptr, nullptr, nullptr,
               &ncnt[b], &fcnt[b], err);
    if ((threadIdx.x & 31) == 0) atomicMax(fmax, fcnt[b]);
}

__global__ void __launch_bounds__(32 * MB_WARPS) k_mb_emit(int NP, int W, int M, int nb, const int32_t *m_large,
                                                          const int2 *m_small, const int32_t *m_info,
                                                          const int *first, const int *second, const int *noff,
                                                          const int *foff, int32_t *mn_node, int2 *mn_slot,
                                                          int32_t *mb_foreign, int *err) {
    __shared__ int cand[MB_WARPS][FCAP], keep[MB_WARPS][FCAP], cnt[MB_WARPS][2];
    const int w = threadIdx.x >> 5, b = blockIdx.x * MB_WARPS + w;
    if (b >= nb) return;
    warp_block(NP, W, M, b, m_large, m_small, m_info, first, second, cand[w], keep[w], mn_node + noff[b],
               mn_slot + noff[b], mb_foreign + foff[b], &cnt[w][0], &cnt[w][1], err);
}

// The area of the leaves and the large-face length of the mortars, each
// summed in a fixed order (one block; thread t takes every 1024th entry from
// t, then a tree over the threads), so a mesh always gives the same bits.
__global__ void __launch_bounds__(1024) k_totals(const RemeshMesh Md, const int8_t *lev, int K, const int32_t *m_large,
                                                 const int32_t *m_info, int M, double *out) {
    __shared__ double sa[1024], sl[1024], hx[25], hy[25];
    const int t = threadIdx.x;
    if (t < 25) {   // element sides per level, formed as the geometry forms them
        hx[t] = (Md.x1 - Md.x0) / ((double)Md.nx0 * (double)(1LL << t));
        hy[t] = (Md.y1 - Md.y0) / ((double)Md.ny0 * (double)(1LL << t));
    }
    __syncthreads();
    double a = 0.0, l = 0.0;
    for (int e = t; e < K; e += 1024) {
        const int v = lev[e];
        a += hx[v] * hy[v];
    }
    for (int m = t; m < M; m += 1024) {
        const int v = lev[m_large[m]];
        l += (m_info[m] & 1) == 0 ? hy[v] : hx[v];
    }
    sa[t] = a;
    sl[t] = l;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (t < h) { sa[t] += sa[t + h]; sl[t] += sl[t + h]; }
        __syncthreads();
    }
    if (t == 0) { out[0] = sa[0]; out[1] = sl[0]; }
}

}  // namespace rm

// ------------------------------------------------------ host drivers ----
namespace {
int grid_for(long long n, int num_sms) {
    return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)num_sms * 16));
}
template <typename T>
cudaError_t read1(const T *d, T *h, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(h, d, sizeof(T), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}
}  // namespace

size_t remesh_plan_scratch_ints(int K) {
    // mark x2, cnt, fcnt, off (K + 1), foff (K + 1), err/changed, scan temporaries
    return (size_t)6 * (K + 2) + rm::scan_tmp_ints(K) + 16;
}

cudaError_t remesh_plan(const PlanIn &in, PlanOut &out, int *scratch, cudaStream_t st, int num_sms, int *K_new,
                        int *n_fam, int *iterations) {
    const int K = in.K;
    int *mark = scratch, *mark2 = mark + (K + 2), *cnt = mark2 + (K + 2), *fcnt = cnt + (K + 2);
    int *off = fcnt + (K + 2), *foff = off + (K + 2), *flags = foff + (K + 2), *tmp = flags + 8;
    const int g = grid_for(K, num_sms);
    rm::k_marks<<<g, 256, 0, st>>>(in.ind, in.lev, K, in.refine, in.coarsen, in.min_level, in.max_level, mark2);
    rm::k_family<<<g, 256, 0, st>>>(in.fnbr, in.ftype, in.ix, in.iy, K, mark2, mark);
    int it = 0;
    // sweeps in batches of four, one host read per batch: a sweep after the
    // fixed point changes nothing, and the first sweep that changed nothing
    // ends the loop
    constexpr int B = 4;
    for (bool more = true; more;) {
        cudaMemsetAsync(flags, 0, sizeof(int) * B, st);
        for (int k = 0; k < B; ++k)
            rm::k_balance<<<g, 256, 0, st>>>(in.fnbr, in.ftype, in.m_large, in.m_small, in.lev, in.ix, in.iy, K, mark,
                                             flags + k);
        int ch[B];
        cudaError_t e = cudaMemcpyAsync(ch, flags, sizeof(ch), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        more = false;
        for (int k = 0; k < B; ++k) {
            ++it;
            if (!ch[k]) break;
            if (k == B - 1) more = true;
        }
        if (more && it >= 64) {   // 2:1 balance propagates over the levels only: not reached on a valid mesh
            *iterations = -1;
            return cudaSuccess;
        }
    }
    *iterations = it;
    rm::k_emit_count<<<g, 256, 0, st>>>(in.fnbr, in.ftype, in.ix, in.iy, K, mark, cnt, fcnt);
    rm::exclusive_scan(cnt, off, K, tmp, st);
    rm::exclusive_scan(fcnt, foff, K, tmp, st);
    int kn = 0, nf = 0;
    cudaError_t e = cudaMemcpyAsync(&kn, off + K, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nf, foff + K, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *K_new = kn;
    *n_fam = nf;
    if (kn > out.capacity) return cudaSuccess;   // the caller's buffers are too small
    rm::k_emit<<<g, 256, 0, st>>>(in.fnbr, in.ftype, in.lev, in.ix, in.iy, K, mark, off, foff, out.lev, out.ix,
                                  out.iy, out.kind, out.src, out.fam);
    return cudaGetLastError();
}

size_t remesh_build_scratch_bytes(int K, int NP) {
    int cap = 1;
    while (cap < 2 * K) cap <<= 1;
    const size_t k4 = (size_t)4 * K + 2;
    return sizeof(unsigned long long) * cap + sizeof(int) * cap        // hash table
           + sizeof(int) * (2 * k4 + 16) + sizeof(int2) * k4           // mortar flags, offsets, candidates
           + sizeof(int) * 2 * (size_t)K * NP * NP                     // first / second slot per node
           + sizeof(int) * (size_t)rm::scan_tmp_ints((int)k4) + 4096;
}

cudaError_t remesh_build_faces(const BuildIn &in, BuildOut &out, void *scratch, cudaStream_t st, int num_sms,
                               int *M_new, int *err_bits) {
    const int K = in.K;
    int cap = 1;
    while (cap < 2 * K) cap <<= 1;
    char *p = (char *)scratch;
    unsigned long long *keys = (unsigned long long *)p; p += sizeof(unsigned long long) * cap;
    int *vals = (int *)p; p += sizeof(int) * cap;
    const size_t k4 = (size_t)4 * K + 2;
    int *mflag = (int *)p; p += sizeof(int) * k4;
    int *moff = (int *)p; p += sizeof(int) * k4;
    int *err = (int *)p; p += sizeof(int) * 16;
    int2 *cand = (int2 *)p; p += sizeof(int2) * k4;
    int *tmp = (int *)p;
    const int g = grid_for(K, num_sms), g4 = grid_for(4LL * K, num_sms);
    cudaMemsetAsync(err, 0, sizeof(int), st);
    rm::k_hash_clear<<<grid_for(cap, num_sms), 256, 0, st>>>(keys, cap);
    rm::k_hash_insert<<<g, 256, 0, st>>>(in.lev, in.ix, in.iy, K, keys, vals, cap - 1, err);
    rm::k_geom<<<g, 256, 0, st>>>(in.mesh, in.lev, in.ix, in.iy, K, out.geom, out.geoc, out.sim);
    rm::k_faces<<<g4, 256, 0, st>>>(in.mesh, in.lev, in.ix, in.iy, K, keys, vals, cap - 1, out.fnbr, out.ftype, mflag,
                                    cand, err);
    rm::exclusive_scan(mflag, moff, 4 * K, tmp, st);
    int m = 0, eb = 0;
    cudaError_t e = cudaMemcpyAsync(&m, moff + 4 * K, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&eb, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *M_new = m;
    *err_bits = eb;
    if (eb || m > out.capM) return cudaSuccess;
    rm::k_mortars<<<g4, 256, 0, st>>>(mflag, moff, cand, K, out.fnbr, out.ftype, out.m_large, out.m_small, out.m_info);
    rm::k_check_pending<<<g4, 256, 0, st>>>(out.ftype, K, err);
    e = read1(err, &eb, st);
    if (e != cudaSuccess) return e;
    *err_bits = eb;
    return cudaGetLastError();
}

cudaError_t remesh_build_mortar_nodes(const NodesIn &in, NodesOut &out, void *scratch, cudaStream_t st,
                                      int num_sms, int *n_mnodes, int *n_blocks, int *fmax, int *err_bits) {
    const int NP = in.NP, Q = 3 * NP, M = in.M, W = in.W;
    const long long nn = (long long)in.K * NP * NP;
    char *p = (char *)scratch;
    int *first = (int *)p; p += sizeof(int) * nn;
    int *second = (int *)p; p += sizeof(int) * nn;
    const int nb = M > 0 ? (M + W - 1) / W : 0;
    int *ncnt = (int *)p; p += sizeof(int) * (nb + 2);
    int *fcnt = (int *)p; p += sizeof(int) * (nb + 2);
    int *noff = (int *)p; p += sizeof(int) * (nb + 2);
    int *foff = (int *)p; p += sizeof(int) * (nb + 2);
    int *flags = (int *)p; p += sizeof(int) * 16;
    int *tmp = (int *)p;
    *n_blocks = nb;
    cudaMemsetAsync(flags, 0, sizeof(int) * 4, st);
    if (M == 0) {
        *n_mnodes = 0; *fmax = 0; *err_bits = 0;
        cudaMemsetAsync(out.mb_node_off, 0, sizeof(int), st);
        cudaMemsetAsync(out.mb_for_off, 0, sizeof(int), st);
        return cudaGetLastError();
    }
    const int gs = grid_for((long long)M * Q, num_sms);
    rm::k_node_fill<<<grid_for(nn, num_sms), 256, 0, st>>>(first, nn, 0x7fffffff);
    rm::k_node_fill<<<grid_for(nn, num_sms), 256, 0, st>>>(second, nn, 0x7fffffff);
    rm::k_node_first<<<gs, 256, 0, st>>>(NP, M, in.m_large, in.m_small, in.m_info, first);
    rm::k_node_second<<<gs, 256, 0, st>>>(NP, M, in.m_large, in.m_small, in.m_info, first, second, nullptr);
    rm::k_node_third<<<gs, 256, 0, st>>>(NP, M, in.m_large, in.m_small, in.m_info, first, second, flags);
    const int gmb = (nb + rm::MB_WARPS - 1) / rm::MB_WARPS;
    rm::k_mb_count<<<gmb, 32 * rm::MB_WARPS, 0, st>>>(NP, W, M, nb, in.m_large, in.m_small, in.m_info, first, second,
                                                     ncnt, fcnt, flags + 1, flags);
    rm::exclusive_scan(ncnt, noff, nb, tmp, st);
    rm::exclusive_scan(fcnt, foff, nb, tmp, st);
    int hv[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(hv, flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hv + 2, noff + nb, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hv + 3, foff + nb, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *err_bits = hv[0];
    *fmax = hv[1];
    *n_mnodes = hv[2];
    const int nfore = hv[3];
    if (hv[0] || hv[2] > out.cap_nodes || nfore + 1 > out.cap_foreign || nb + 1 > out.cap_blocks) return cudaSuccess;
    rm::k_mb_emit<<<gmb, 32 * rm::MB_WARPS, 0, st>>>(NP, W, M, nb, in.m_large, in.m_small, in.m_info, first, second,
                                                    noff, foff, out.mn_node, out.mn_slot, out.mb_foreign, flags);
    cudaMemcpyAsync(out.mb_node_off, noff, sizeof(int) * (nb + 1), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(out.mb_for_off, foff, sizeof(int) * (nb + 1), cudaMemcpyDeviceToDevice, st);
    if (nfore == 0) cudaMemsetAsync(out.mb_foreign, 0, sizeof(int), st);
    return cudaGetLastError();
}

void remesh_totals(const RemeshMesh &mesh, const int8_t *lev, int K, const int32_t *m_large, const int32_t *m_info,
                   int M, double *out, cudaStream_t st) {
    rm::k_totals<<<1, 1024, 0, st>>>(mesh, lev, K, m_large, m_info, M, out);
}

size_t remesh_nodes_scratch_bytes(int K, int NP, int M, int W) {
    const int nb = M > 0 ? (M + W - 1) / W : 0;
    return sizeof(int) * (2 * (size_t)K * NP * NP + 4 * (size_t)(nb + 2) + 16 + rm::scan_tmp_ints(nb + 2)) + 4096;
}

}  // namespace idp
