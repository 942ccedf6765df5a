// Selection table of the tensor-core Wilson hop (hop_mma.cuh), built at
// compile time.
//
// One hop direction d (d = 2 mu: forward, d = 2 mu + 1: backward) acts on the
// neighbour's 4-spinor psi (12 complex components c = 3 alpha + a) as
//
//   out[beta b] += sum_{alpha a} P_d[beta][alpha] V_d[b][a] psi[alpha a],
//   P_d = 1 - g_mu (forward) or 1 + g_mu (backward),
//   V_d = U_mu(x) (forward) or U_mu(x - mu)^dag (backward),
//
// which in real arithmetic is a 24 x 24 matrix O_d (row 2 o + ro: real part
// ro = 0 or imaginary part ro = 1 of output component o; column 2 n + ri of
// input component n).  For z = P_d[beta][alpha] V_d[b][a]:
//   O_d[2o][2n] = Re z,  O_d[2o][2n+1] = -Im z,
//   O_d[2o+1][2n] = Im z, O_d[2o+1][2n+1] = Re z.
// The hop multiplies O_d with the block of right-hand sides by mma.sync
// m16n8k16 (input components 0..7) and m16n8k8 (components 8..11), in two
// row tiles (output components 0..7 and 8..11).  Lane l = 4 g + t of a warp
// holds, as pairs of bf16 in one 32-bit word, the A-fragment entries of rows
// 2 o + (g & 1) with o in {g >> 1, 4 + (g >> 1), 8 + (g >> 1)} and columns
// 2 n, 2 n + 1 with n in {t, 4 + t, 8 + t}: nine words ("slots", s = 3 i + j
// for the i-th o and j-th n).
//
// Every entry of P_d is 0, +-1 or +-i (chiral DeGrand-Rossi gamma matrices,
// g_mu = [[0, X_mu], [X_mu^dag, 0]] with X_1 = i sigma_x, X_2 = -i sigma_y,
// X_3 = i sigma_z, X_4 = 1), so each slot word is the link element word
// w = (Re u, Im u) (bf16 pair, real part in the low half) with its halves
// possibly exchanged and sign bits possibly flipped, or zero.  The table gives,
// per direction, slot and lane, the byte-permute selector (low 16 bits: 0x3210
// keep, 0x1032 exchange, 0x4444 zero), the byte offset of the link element in
// the direction's nine words (bits 16..23) and the sign mask to exclusive-or,
// as two bits: bit 24 for 0x8000 (low half), bit 25 for 0x80000000 (high
// half); the byte permute reads only the low 16 bits.
#pragma once

#include <stdint.h>

namespace dl {

struct MmaSel {
    uint32_t code[8][9][32];  // [direction][slot][lane]: selector | link byte offset << 16 | sign bits << 24
};

// gamma_mu[r][c] as a power of i: 0 for zero, q + 1 for i^q.
constexpr int mma_gamma_code(int mu, int r, int c) {
    if ((r < 2) == (c < 2)) return 0;
    // X_mu entries as i^q codes: 1 -> 1, i -> 2, -1 -> 3, -i -> 4
    const int x[4][2][2] = {{{0, 2}, {2, 0}}, {{0, 3}, {1, 0}}, {{2, 0}, {0, 4}}, {{1, 0}, {0, 1}}};
    if (r < 2) return x[mu][r][c - 2];
    const int v = x[mu][c][r - 2];  // (X^dag)[r-2][c] = conj(X[c][r-2])
    if (v == 0) return 0;
    return (4 - (v - 1)) % 4 + 1;
}

// P_d[beta][alpha] as a power of i (0: zero entry).
constexpr int mma_p_code(int d, int beta, int alpha) {
    if (beta == alpha) return 1;
    const int gc = mma_gamma_code(d >> 1, beta, alpha);
    if (gc == 0) return 0;
    int q = gc - 1;
    if ((d & 1) == 0) q = (q + 2) % 4;  // 1 - g_mu: times -1
    return q + 1;
}

// A word transform: exchange the halves (swap) then flip the sign bits in mask.
struct MmaXf {
    int swap;
    uint32_t mask;
};
constexpr uint32_t mma_swap_halves(uint32_t m) { return (m >> 16) | (m << 16); }
// first a, then b
constexpr MmaXf mma_compose(MmaXf a, MmaXf b) {
    return MmaXf{a.swap ^ b.swap, (b.swap ? mma_swap_halves(a.mask) : a.mask) ^ b.mask};
}

constexpr MmaSel make_mma_sel() {
    MmaSel T{};
    for (int d = 0; d < 8; ++d)
        for (int lane = 0; lane < 32; ++lane) {
            const int g = lane >> 2, t = lane & 3, ro = g & 1;
            const int os[3] = {g >> 1, 4 + (g >> 1), 8 + (g >> 1)};
            const int ns[3] = {t, 4 + t, 8 + t};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    const int s = 3 * i + j, o = os[i], n = ns[j];
                    uint32_t so = 0x4444u, m = 0u;  // zero word
                    if (o < 12 && n < 12) {
                        const int beta = o / 3, b = o % 3, alpha = n / 3, a = n % 3;
                        const int pc = mma_p_code(d, beta, alpha);
                        if (pc != 0) {
                            const bool bwd = (d & 1) != 0;
                            const int idx = bwd ? 3 * a + b : 3 * b + a;  // V = U (fwd) or U^dag (bwd)
                            MmaXf x{0, bwd ? 0x80000000u : 0u};           // conjugation: negate Im
                            const int q = pc - 1;                          // times i^q: (r, m) -> (-m, r) per step
                            const MmaXf rot[4] = {{0, 0u}, {1, 0x00008000u}, {0, 0x80008000u}, {1, 0x80000000u}};
                            x = mma_compose(x, rot[q]);
                            // row ro = 0: (Re z, -Im z); ro = 1: (Im z, Re z)
                            x = mma_compose(x, ro == 0 ? MmaXf{0, 0x80000000u} : MmaXf{1, 0u});
                            so = (x.swap ? 0x1032u : 0x3210u) | ((uint32_t)(4 * idx) << 16);
                            m = x.mask;
                        }
                    }
                    T.code[d][s][lane] = so | ((m & 0x8000u) ? 1u << 24 : 0u) | ((m & 0x80000000u) ? 1u << 25 : 0u);
                }
        }
    return T;
}

}  // namespace dl
