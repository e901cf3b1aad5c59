// FP64 forward, column and pair-product kernels for transform size 1024.
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<double, 1024>::fwd_rows(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 1024>::fwd_cols(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 1024>::pair_cols(const Geom&, const PipeArgs<double>&, cudaStream_t);
template int Sized<double, 1024>::tm_cols(int);
template cudaError_t Sized<double, 1024>::tm_max_blocks(int*);
}
