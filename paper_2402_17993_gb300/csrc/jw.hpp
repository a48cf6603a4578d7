// Host-side Jordan-Wigner compiler: fermionic operators of Eq. 2 and Eq. 4
// to real Pauli terms in the X^x Z^z form, grouped by X-mask.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "common.hpp"

namespace uccsd {

// c * X^x Z^z, acting as X^x Z^z |y> = (-1)^{popc(y & z)} |y ^ x>.
struct XZTerm {
    uint32_t x, z;
    double c;
};

struct CompiledH {
    int n_qubits = 0;
    int n_terms = 0;                    // nonzero Pauli terms after merging
    std::vector<XZTerm> terms;          // sorted by (x, z)
    std::vector<GroupT<double>> groups; // off-diagonal groups (nb = 2 or 4)
    std::vector<double> spec;           // spectator rows [w][pat] (4 per row), n_qubits rows per 2-bit group
    // diagonal group as an occupation quadratic form
    double c0 = 0.0;
    std::vector<double> diag_a;         // n
    std::vector<double> diag_b;         // n*n, upper triangle q < r used
    bool has_diag = false;
};

// Compile Eq. 2 (spin-orbital integrals from spatial h, eri) under the
// Jordan-Wigner mapping.  Returns false and sets err on failure.
bool compile_hamiltonian(int n_orb, const double *h, const double *eri, double e_core,
                         CompiledH *out, std::string *err);

// Merged X^x Z^z terms of Eq. 2 with spin orbital P on qubit qubit_of[P]
// (Jordan-Wigner strings follow the qubit order), sorted by (x, z).
bool pauli_terms_ordered(int n_orb, const double *h, const double *eri, double e_core,
                         const int *qubit_of, std::vector<XZTerm> *out, std::string *err);

// Generator G = tau - tau^dag of one excitation row (i, j, a, b) in the
// X^x Z^z form, reduced to (flip mask, occupied-side mask, Jordan-Wigner
// parity mask, sign s0) so that G|x> = s0 (-1)^{popc(x & par)} |x ^ flip>
// for x with the occupied-side pattern.
struct CompiledExc {
    uint32_t flip, occ, par;
    int s0;
    int nb;
};
bool compile_excitation(int n_qubits, const int32_t *row, CompiledExc *out, std::string *err);

// Tapered symmetry-conserving Bravyi-Kitaev positions of the sector
// determinants (tapering.cpp): determinant (alpha string sa, beta string sb)
// at aoff[sa] + boff[sb] of the 2^(2 n_orb - 2) vector, in the qubit order of
// uccsd_pauli_terms_scbk.
void scbk_addresses(int n_orb, std::vector<uint32_t> *aoff, std::vector<uint32_t> *boff);

}  // namespace uccsd
