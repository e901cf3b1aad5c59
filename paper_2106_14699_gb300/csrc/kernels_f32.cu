// FP32-transform instantiation of the CMIF launch sequence.
#define CMIF_DEFINE_TM_HELPERS 1  // the TMEM row-kernel helpers live in this translation unit
#include "pipeline_impl.cuh"
namespace cmif {
CMIF_INSTANTIATE(float)
}
