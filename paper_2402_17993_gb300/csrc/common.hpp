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
    R lut[16];
};

// One factor exp(angle * G) of the Trotter schedule, in the local bit space
// of the shared-memory tile of the run that applies it.  For a basis state
// x with the occupied-side pattern (occ bits set, the other flip bits
// clear) and partner x' = x ^ flip:
//   G|x>  = s(x)|x'>,   G|x'> = -s(x)|x>,
//   s(x)  = s0 * (-1)^{popc(x_local & par_l) + popc(x_rest & par_rest)}.
struct OpDev {
    uint32_t flip_l;    // flipped bits (tile-local positions)
    uint32_t occ_l;     // bits that are occupied on the x side (local)
    uint32_t par_l;     // Jordan-Wigner parity mask inside the tile (local)
    uint32_t par_rest;  // Jordan-Wigner parity mask outside the tile (global bits)
    int32_t nb;         // 2 (single) or 4 (double)
    int32_t pos[4];     // flipped local bit positions, ascending
    int32_t s0;         // +1 or -1
    int32_t op;         // index of this factor in the schedule
};

// A shared-memory pass: the factors [op_begin, op_end) of the schedule all
// flip only bits inside the tile bit set `tmask` (L bits, containing the
// low bits 0..c-1), so every tile of 2^L amplitudes evolves on its own.
struct RunDev {
    uint32_t tmask;     // tile bits (global positions)
    uint32_t rmask;     // the other bits
    int32_t L;          // popcount(tmask)
    int32_t c;          // contiguous low bits in tmask
    int32_t op_begin, op_end;  // range in the run's op table
};

}  // namespace uccsd
