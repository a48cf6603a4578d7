// Shared host/device data layouts of the UCCSD library.
#pragma once
#include <cstdint>

namespace uccsd {

// One X-mask group of the Jordan-Wigner Hamiltonian (Eq. 2 mapped to
// qubits).  All Pauli terms of a group flip the same bits `xmask`, so
//   (H psi)[x] = sum_g f_g(x ^ xmask_g) psi[x ^ xmask_g]
// with f_g(y) = (-1)^{popc(y & jmask)} * ( lut[pat(y)]
//                                          + sum_{w in occ(y), w not in xmask} spec[w][pat(y)] )
// where pat(y) collects y's bits at pos[0..nb) (bit k = bit pos[k] of y).
// nb = 0 marks the diagonal group, evaluated from the occupation quadratic
// form c0 + sum_q a_q y_q + sum_{q<r} b_qr y_q y_r instead.
template <typename R>
struct GroupT {
    uint32_t xmask;
    uint32_t jmask;
    int32_t nb;        // 0, 2 or 4 flipped bits
    int32_t spec;      // offset into the spectator table (rows of 4), -1 = none
    uint32_t active;   // bit p set: pattern p conserves N_alpha and N_beta
    int32_t pos[4];    // flipped bit positions, ascending
    // Flip bits inside the H-apply tile (the low LH bits) as alpha / beta
    // string masks (alpha string bit k = qubit 2k, beta string bit k =
    // qubit 2k+1), and the occupied flip bits an active source pattern
    // has among the alpha / beta flip bits (half of them).
    uint32_t mla, mlb;
    int32_t ha, hb;
    R lut[16];
};

// H-apply tables by group class.  Orbital strings: bit t of an alpha
// string is qubit 2t, bit t of a beta string is qubit 2t+1.  Pair index of
// orbitals p < q: q(q-1)/2 + p; quad index of p < q < r < s:
// C(s,4) + C(r,3) + C(q,2) + p.  j packs the Jordan-Wigner interval mask of
// the group as (alpha string) | (beta string) << 16.  Absent groups have
// zero tables.
//
// Mixed group (alpha pair, beta pair): lut[asel + 2 bsel] is f_g at the
// source y that occupies the higher (asel = 1) or lower alpha orbital of the
// pair and the higher (bsel = 1) or lower beta orbital.
template <typename R>
struct MixT {
    R lut[4];
    uint32_t j;
};
// The same mixed groups by ordered excitation: entry ((p n + q) n + j) n + b
// of an n_orb^4 array holds, for a target with alpha p occupied and q empty
// and beta j occupied and b empty (the source flips both pairs), the LUT
// value of that source pattern and the group's Jordan-Wigner mask.
template <typename R>
struct alignas(sizeof(R) == 4 ? 8 : 16) MixO {
    R w;
    uint32_t j;
};
// One alpha double excitation of an H-apply row, staged per CTA: the
// same-spin double's table value, the source row offset, the source alpha
// string and the group's Jordan-Wigner mask.
template <typename R>
struct ADbl {
    R w;
    uint32_t xoff, s, j;
};
// Same-spin single (pair): lut[sel] at the source occupying the higher
// (sel = 1) or lower orbital; spectator rows start at spec (rows of 4,
// pattern 1 = lower occupied, 2 = higher occupied).
template <typename R>
struct SglT {
    R lut[2];
    uint32_t j;
    int32_t spec;
};
// Same-spin double (quad): lut[pattern of the source over the sorted quad].
template <typename R>
struct DblT {
    R lut[16];
    uint32_t j;
};

// A shared-memory pass over compact sector tiles.  The factors
// [op_begin, op_end) of the schedule flip only bits inside the tile bit set
// `tmask`, so every tile (fixed values of the other bits) evolves on its
// own.  A tile keeps only its electron-sector entries: with (a, b) the
// alpha/beta electrons the sector leaves for the tile bits, the entries
// form a dense [C(La, a)] x [C(Lb, b)] array indexed by the ranks of the
// tile's alpha and beta bit strings among the strings of the same
// popcount.  Amplitudes outside the sector are zero and never touched.
struct CRunDev {
    uint32_t tmask;      // tile bits (global positions)
    uint32_t rmask;      // the other bits
    int32_t La, Lb;      // alpha / beta bits of the tile
    int32_t op_begin, op_end;
    int32_t spread_off;  // run's spread table: 2^La alpha then 2^Lb beta entries
    int32_t n_tiles;     // 2^(n - La - Lb)
    int32_t max_entries; // largest compact tile over the run's CTAs
    int32_t max_da, max_db;  // largest C(La, a), C(Lb, b) over the run's CTAs
    int32_t pl_base;     // precomputed pair lists: first (offset, count) entry of the run, or -1
    int32_t emap_base;   // entry maps: first entry of the run's tiles (max_entries each), or -1
};

// One factor exp(angle * G) of the schedule in the string spaces of its
// run's tile (bit k of an alpha string = the k-th alpha bit of the tile).
// The occupied side of a pair has the bits oa/ob set and the other flip
// bits clear; the partner flips fa/fb.  JW sign of the pair:
//   s0 * (-1)^{popc(sa & pa) + popc(sb & pb) + popc(rest & par_rest)}.
// op_s0: index of the factor in the schedule, bit 31 set when s0 = -1.
struct COpDev {
    uint32_t fa, fb;      // flipped bits
    uint32_t oa, ob;      // occupied-side bits
    uint32_t pa, pb;      // Jordan-Wigner parity bits inside the tile
    uint32_t par_rest;    // Jordan-Wigner parity bits outside the tile (global)
    uint32_t op_s0;
};

}  // namespace uccsd
