// FP32 forward, column and pair-product kernels for transform size 2048.
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<float, 2048>::fwd_rows(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 2048>::fwd_cols(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 2048>::pair_cols(const Geom&, const PipeArgs<float>&, cudaStream_t);
template int Sized<float, 2048>::tm_cols(int);
template cudaError_t Sized<float, 2048>::tm_max_blocks(int*);
}
