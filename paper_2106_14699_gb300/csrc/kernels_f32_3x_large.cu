// FP32 forward, column and pair-product kernels for the transform sizes 1536, 3072 (3 * 2^k).
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<float, 1536>::fwd_rows(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 1536>::fwd_cols(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 1536>::pair_cols(const Geom&, const PipeArgs<float>&, cudaStream_t);
template int Sized<float, 1536>::tm_cols(int);
template cudaError_t Sized<float, 1536>::tm_max_blocks(int*);
template cudaError_t Sized<float, 1536>::pair_rows_w(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 1536>::rows_w_smem();
template cudaError_t Sized<float, 1536>::rows_w_max_blocks(int*);
template cudaError_t Sized<float, 3072>::fwd_rows(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 3072>::fwd_cols(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 3072>::pair_cols(const Geom&, const PipeArgs<float>&, cudaStream_t);
template int Sized<float, 3072>::tm_cols(int);
template cudaError_t Sized<float, 3072>::tm_max_blocks(int*);
template cudaError_t Sized<float, 3072>::pair_rows_w(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 3072>::rows_w_smem();
template cudaError_t Sized<float, 3072>::rows_w_max_blocks(int*);
}
