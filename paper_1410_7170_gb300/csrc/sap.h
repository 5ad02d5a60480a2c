// Schwarz alternating procedure (internal interface).
#pragma once
#include "internal.h"

namespace ovl {

struct SapGeom {
    int b[4];        // block extent per direction
    int nblk[4];     // blocks per direction
    int stride[4];   // local lexicographic strides inside a block
    int nb;          // sites per block
    int tps;         // threads per site of the FP32 block kernel (1, 2 or 4; FP64 uses 1)
};

inline SapGeom make_sap_geom(const Geom &g, const int b[4]) {
    SapGeom s;
    for (int m = 0; m < 4; m++) {
        s.b[m] = b[m];
        s.nblk[m] = g.L[m] / b[m];
    }
    s.stride[3] = 1;
    s.stride[2] = b[3];
    s.stride[1] = b[3] * b[2];
    s.stride[0] = b[3] * b[2] * b[1];
    s.nb = b[0] * b[1] * b[2] * b[3];
    s.tps = 1;
    return s;
}

// x = M_SAP v: `cycles` multiplicative Schwarz cycles from x = 0 on D_W(m0), block
// solves by mr_iters minimal-residual steps. r is a scratch spinor.
cudaError_t sap_f32(const Geom &g, const SapGeom &sg, const float4 *U, const float4 *v, float4 *x, float4 *r,
                    float m0, int cycles, int mr_iters, cudaStream_t st);
cudaError_t sap_f64(const Geom &g, const SapGeom &sg, const double2 *U, const double2 *v, double2 *x, double2 *r,
                    double m0, int cycles, int mr_iters, cudaStream_t st);

}  // namespace ovl
