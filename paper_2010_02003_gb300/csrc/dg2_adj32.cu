// dg2_adj32.cu -- the discrete adjoint of dg2_adj.cu with FP32 storage: the same
// source compiled with float as the type of every device buffer (state,
// checkpoints, operator adjoints, face Jacobians, gradients), in namespace
// dg2::adj32.  Arithmetic stays FP64 in registers: the depth-form operators of
// Eqs. 4-5 cancel the hydrostatic pressure against the bed term only to the
// working precision, and in FP32 that residue drives spurious flows larger than
// the misfit signal of a calibration (the forward FP32 path avoids it with its
// free-surface form).  What FP32 storage buys is half the memory of the
// checkpointed states, so twice the snapshots fit.
#define DG2_ADJ_STORE float
#define DG2_ADJ_NS adj32
// arithmetic type of this translation unit (FP64; DG2_ADJ32_ARITH=float compiles an
// all-FP32 variant, which measured unusable for calibration: the hydrostatic
// pressure and bed term of Eqs. 4-5 cancel only to working precision)
#ifdef DG2_ADJ32_ARITH
#define DG2_ADJ_ARITH DG2_ADJ32_ARITH
#endif
#include "dg2_adj.cu"
