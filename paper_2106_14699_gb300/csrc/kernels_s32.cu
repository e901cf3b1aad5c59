// Two-term FP32 (split-precision) instantiation of the CMIF launch sequence.
#include "pipeline_impl.cuh"
namespace cmif {
CMIF_INSTANTIATE(df32)
}
