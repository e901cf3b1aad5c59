// FP64 forward, column, pair-product and weighted-row kernels for transform size 4096.
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<double, 4096>::fwd_rows(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 4096>::fwd_cols(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 4096>::pair_cols(const Geom&, const PipeArgs<double>&, cudaStream_t);
template int Sized<double, 4096>::tm_cols(int);
template cudaError_t Sized<double, 4096>::tm_max_blocks(int*);
template cudaError_t Sized<double, 4096>::pair_rows_w(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 4096>::rows_w_smem();
template cudaError_t Sized<double, 4096>::rows_w_max_blocks(int*);
}
