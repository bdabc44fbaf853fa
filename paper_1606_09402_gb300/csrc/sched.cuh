// Work schedule of the tensor-core passes over A (integer logic only, host and device).
//
// A pass computes D (M x N) = sum over K of A-tile x V-tile products.  D is cut into units of
// TC_BM x bn (tiles_m x tiles_n), each with kb k-blocks of TC_BK.  A launch of G persistent CTAs
// walks the units in one of three ways:
//   raster   (streamk 0): CTA c runs whole units c, c + G, c + 2G, ...;
//   stream-K (streamk 1): the flattened (unit, k-block) sequence of all units is split into G
//                         even ranges, one per CTA;
//   hybrid   (streamk 2): the first dp_units units (whole waves) in raster order, then the
//                         flattened k-blocks of the remaining units split into G even ranges.
// A split range leaves at most two partial units per CTA: its first segment goes to partial slot
// 0, its last to slot 1, and whole units in between are written directly.  The fix-up sums, for
// every unit of the split space that more than one CTA touched, the partial slots of those CTAs
// in CTA order.  SegWalk (the kernels) and split_owners / split_slot (the fix-up) must agree;
// tests/sched_check.cu verifies that they do over many shapes, on the host.
#pragma once

#include <algorithm>
#include <cstdint>

namespace qb {

constexpr int TC_BM = 128;          // rows of a unit (the MMA M)
constexpr int TC_BK = 64;           // k per k-block
constexpr int TC_MAX_SK_CTAS = 160; // split launches use at most this many CTAs

struct Sched {
    int tiles_m, tiles_n, kb;   // units = tiles_m * tiles_n, k-blocks per unit
    int streamk;                // 0 raster, 1 stream-K, 2 hybrid
    int dp_units;               // hybrid: units run whole before the split tail
};
// Segment of a CTA: unit u, k-blocks [k0, k1), slot = partial slot (-1 = whole unit)
struct Seg {
    int u, k0, k1, slot;
};
__host__ __device__ inline int64_t sk_begin(int64_t total, int64_t c, int64_t G) {
    return (total * c) / G;
}

// The segments of CTA cta, in order; every warp role of the CTA walks the same sequence.
struct SegWalk {
    const Sched* sc;
    int64_t pos, end, tail_beg, tail_end;
    int G;
    bool first, split;
    __host__ __device__ SegWalk(const Sched& s, int cta, int g) : sc(&s), G(g), first(true) {
        const int64_t units = int64_t(s.tiles_m) * s.tiles_n;
        tail_beg = tail_end = 0;
        if (s.streamk == 1) {
            pos = sk_begin(units * s.kb, cta, G);
            end = sk_begin(units * s.kb, cta + 1, G);
            split = true;
        } else {
            pos = cta;
            end = s.streamk == 2 ? s.dp_units : units;
            split = false;
            if (s.streamk == 2) {
                const int64_t t0 = int64_t(s.dp_units) * s.kb;
                const int64_t tt = (units - s.dp_units) * s.kb;
                tail_beg = t0 + sk_begin(tt, cta, G);
                tail_end = t0 + sk_begin(tt, cta + 1, G);
            }
        }
    }
    __host__ __device__ bool next(Seg& sg) {
        if (!split && pos >= end) {
            if (sc->streamk != 2 || tail_beg >= tail_end) return false;
            split = true;                  // raster units done: this CTA's share of the tail
            first = true;
            pos = tail_beg;
            end = tail_end;
        }
        if (pos >= end) return false;
        if (split) {
            const int64_t u = pos / sc->kb;
            const int k0 = int(pos - u * sc->kb);
            const int64_t rem = end - u * sc->kb;
            const int k1 = int(rem < sc->kb ? rem : int64_t(sc->kb));
            const bool whole = (k0 == 0 && k1 == sc->kb);
            sg = Seg{int(u), k0, k1, whole ? -1 : (first ? 0 : 1)};
            pos = u * sc->kb + k1;
        } else {
            sg = Seg{int(pos), 0, sc->kb, -1};
            pos += G;
        }
        first = false;
        return true;
    }
};

// Units of the split space (the fix-up's grid) and the first of them.
__host__ __device__ inline int split_units(const Sched& s) {
    const int units = s.tiles_m * s.tiles_n;
    return s.streamk == 2 ? units - s.dp_units : units;
}
__host__ __device__ inline int split_first_unit(const Sched& s) {
    return s.streamk == 2 ? s.dp_units : 0;
}
// The CTAs that touched unit ur of the split space: c_first .. c_first + count - 1, count = 0
// when a single CTA covered the whole unit (it wrote the unit directly).
__host__ __device__ inline void split_owners(const Sched& s, int64_t ur, int G, int64_t& c_first,
                                             int& count) {
    const int64_t total = int64_t(split_units(s)) * s.kb;
    auto owner = [&](int64_t x) {
        int64_t c = (x * G) / total;
        while (c + 1 < G && sk_begin(total, c + 1, G) <= x) ++c;
        while (c > 0 && sk_begin(total, c, G) > x) --c;
        return c;
    };
    const int64_t f = ur * s.kb;
    const int64_t a = owner(f), b = owner(f + s.kb - 1);
    c_first = a;
    count = a == b ? 0 : int(b - a + 1);
}
// The partial slot in which CTA c left its part of unit ur: 0 if the unit holds the start of
// c's range, else 1.
__host__ __device__ inline int split_slot(const Sched& s, int64_t ur, int64_t c, int G) {
    const int64_t total = int64_t(split_units(s)) * s.kb;
    return (sk_begin(total, c, G) / s.kb == ur) ? 0 : 1;
}

inline int64_t sched_cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// The schedule of a pass with D = M x N, reduction K, column tile bn, on G SMs.
inline Sched make_sched(int64_t M, int64_t N, int64_t K, int bn, int G) {
    Sched s;
    s.tiles_m = int(sched_cdiv(M, TC_BM));
    s.tiles_n = int(sched_cdiv(N, bn));
    s.kb = int(sched_cdiv(K, TC_BK));
    const int64_t units = int64_t(s.tiles_m) * s.tiles_n;
    // Stream-K balances the k-blocks exactly but costs a fix-up launch and partial-tile traffic
    // (worth about 8 k-blocks of the kernel itself); raster runs whole units in ceil(units / G)
    // waves.  Stream-K is taken for at most one wave of units (a few units with a long k, such
    // as the Q^T Y products of the projections) when it beats raster.  Above one wave it would
    // split up to G units, and every one of them goes through the fix-up: measured on the
    // 40000 x 20000 step, the 157- and 313-unit projection products ran 1.6 ms faster in all
    // (43.7 -> 42.1 ms) as raster or hybrid, which splits only the partial last wave.
    const int64_t waves = (units + G - 1) / G;
    s.streamk = (units <= G && (units * s.kb) / G + 8 < waves * s.kb) ? 1 : 0;
    s.dp_units = 0;
    // Raster with a partial last wave: run the full waves as they are and split only the
    // remaining units' k-blocks across all CTAs (about 17% of a 4.1-wave pass).  Consecutive
    // units of the tail (the column tiles of a row tile) go to CTAs that walk the same k range
    // at the same time, so they still share A through L2.
    // Every CTA must own a non-empty share of the tail (at least G tail k-blocks), or the
    // fix-up would count CTAs that wrote nothing.  Taken only when it saves at least 1/8 of the
    // raster time: a split tail loses some of raster's L2 sharing and adds a fix-up, which
    // measurably outweighs a saving of ~1% (a 27-wave pass) but not one of ~15% (4 waves).
    const int Gs = std::min(G, TC_MAX_SK_CTAS);
    if (!s.streamk && units > Gs && units % Gs != 0) {
        const int64_t full = units / Gs;
        const int64_t rest = units - full * Gs;
        const int64_t t_raster = (full + 1) * s.kb;
        const int64_t t_hybrid = full * s.kb + (rest * s.kb + Gs - 1) / Gs + 8;
        if (rest * s.kb >= Gs && 8 * (t_raster - t_hybrid) > t_raster) {
            s.streamk = 2;
            s.dp_units = int(full * Gs);
        }
    }
    return s;
}

// CTAs to launch: never more than there are k-blocks (stream-K) or units (raster), so that every
// CTA of a stream-K launch owns a non-empty range; a hybrid launch uses exactly the CTA count its
// raster part was planned for.
inline int grid_size(const Sched& s, int sms) {
    const int64_t units = int64_t(s.tiles_m) * s.tiles_n;
    if (s.streamk == 2) return std::min(sms, TC_MAX_SK_CTAS);
    const int64_t work = s.streamk ? units * s.kb : units;
    const int64_t cap = s.streamk ? std::min(sms, TC_MAX_SK_CTAS) : sms;
    return int(std::max<int64_t>(1, std::min<int64_t>(cap, work)));
}

}  // namespace qb
