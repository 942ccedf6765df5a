// Clover (Sheikholeslami-Wohlert) term: M = A - kappa D with the site-local
//
//   A(x) = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x),
//   sigma_{mu nu} = (i/2) [g_mu, g_nu],  F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dag) / (8 i),
//
// Q_{mu nu}(x) the four plaquette leaves of the mu-nu plane at x.  The paper
// uses plain Wilson fermions (Sec. 2); this is the library's optional
// extension, off unless dl_set_clover sets c_sw != 0.  In the chiral basis
// every sigma_{mu nu} is block-diagonal in the spin pairs (0, 1) and (2, 3),
// so A is two hermitian 6 x 6 blocks per site (rows and columns 3 s + a within
// a block).  Layout of A and A^-1: [parity][cb][block][6][6] complex.
//
// With clover the even-odd solve uses the asymmetric Schur system
//   A_ee^-1 Mhat = 1 - kappa^2 A_ee^-1 D_eo A_oo^-1 D_oe,
// so every inner Wilson hop multiplies its result by A^-1 of its output site
// (clover_inv_apply in the hop epilogue) and the outer defect-correction
// steps apply A or A^-1 site by site.  The blocks are built, and applied to
// FP64 fields, by the kernels of clover.cu.
#pragma once

#include "common.cuh"

namespace dl {

struct SigmaBlocks {
    double2 s[6][2][2][2];  // [plane mu<nu][block][row][col] of sigma_{mu nu}
};

// acc <- A^-1 acc at one site (A^-1 in storage S: [2 blocks][6][6] complex).
template <typename S, typename T>
__device__ __forceinline__ void clover_inv_apply(const S *m, cx<T> (&acc)[12]) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        cx<T> v[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) v[j] = acc[6 * b + j];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            cx<T> o = zero<T>();
#pragma unroll
            for (int j = 0; j < 6; ++j) cmac(o, ld_link<S>(m + 2 * (b * 36 + i * 6 + j)), v[j]);
            acc[6 * b + i] = o;
        }
    }
}

}  // namespace dl
