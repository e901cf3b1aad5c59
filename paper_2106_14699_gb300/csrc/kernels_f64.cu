// FP64-transform instantiation of the CMIF launch sequence.
#include "pipeline_impl.cuh"
namespace cmif {
CMIF_INSTANTIATE(double)
}
