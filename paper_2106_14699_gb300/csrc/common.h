// Shared host/device definitions of the CMIF library (not part of the C ABI).
#pragma once
#include <cstdint>

namespace cmif {

// Device-side status word, one per plan; read back by cmif_get_status().
struct DevStatus {
    unsigned flags;        // STATUS_* bits below
    unsigned res_bits[2];  // max |c - round(c)| seen, as float bits: [0] FP32 pass, [1] FP64 pass
    int max_n;             // max_chi N(chi) of the last map (for the gamma gate of Alg. 1)
    int escalations;       // CMIF_AUTO: label pairs re-run in the second precision after the FP32 guard breached
    int predicted;         // CMIF_AUTO: label pairs the precision predicate sent to the second precision up front
    int pad[2];
    unsigned long long max_nw_bits;  // weighted maps (SWMI): max N(chi) as double bits (N >= 0)
};
enum : unsigned {
    STATUS_LABEL_RANGE = 1u,  // a label under mask 1 lies outside [0, K)
    STATUS_PRECISION = 2u,    // residual guard breached in the final precision
    STATUS_TIMEOUT = 4u,      // a bounded device wait gave up
    STATUS_ESCALATE = 8u,     // AUTO: FP32 residual breached, FP64 pass is authoritative
};

// Problem geometry of one CMIF map.
struct Geom {
    int HA, WA, HB, WB;  // image sizes
    int KA, KB;          // label counts
    int R, C;            // output map rows / cols: H_A+H_B-1, W_A+W_B-1
    int P, Q;            // transform sizes (powers of two >= R, C)
    int Qh;              // Q/2 + 1 half-spectrum columns
    int Qs;              // padded row stride (complex elements) of row-major spectra
    // Search window of the call: output rows [r0, r1) are computed, and X_S is
    // rows [r0, r1) x columns [c0, c1) (max N and the peak are taken over it).
    // The whole map unless Alg. 1's padded window is on.
    int r0, r1, c0, c1;
    // Volumes (D_A x H_A x W_A and D_B x H_B x W_B, Sec. 3.1 for n = 3): the
    // slices are transformed as images; Dz = D_A + D_B - 1 depth offsets, R2 =
    // H_A + H_B - 1 rows per depth offset, and the maps have R = Dz * R2 rows
    // (depth-offset major).  Images: DA = DB = Dz = 1, R2 = R.
    int DA, DB, Dz, R2;
    // Units: several floating images against one A in one launch per stage (the
    // rotation angles of Alg. 1).  Unit u's B planes are label * DB + u (DB = units),
    // its map rows u * R2 + (row), R = units * R2; r0, r1 bound the rows of each
    // unit.  1 for a single map (and for volumes).
    int units;
};

constexpr float kResidualGuard = 0.25f;  // a count whose pre-rounding residual reaches this is not trusted
constexpr int kFixBits = 23;             // fixed-point scale of sum c*log2(c): units of 2^-23

}  // namespace cmif
