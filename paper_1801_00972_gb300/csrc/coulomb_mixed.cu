// The float (mixed-precision) Coulomb collision pass: the same source as
// coulomb.cu, compiled as its own unit with fused multiply-add allowed.
#define PIC_COUL_MIXED 1
#include "coulomb.cu"
