// FP32 forward, column and pair-product kernels for the transform sizes 96, 192, 384, 768 (3 * 2^k).
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<float, 96>::fwd_rows(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 96>::fwd_cols(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 96>::pair_cols(const Geom&, const PipeArgs<float>&, cudaStream_t);
template int Sized<float, 96>::tm_cols(int);
template cudaError_t Sized<float, 96>::tm_max_blocks(int*);
template cudaError_t Sized<float, 96>::pair_rows_w(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 96>::rows_w_smem();
template cudaError_t Sized<float, 96>::rows_w_max_blocks(int*);
template cudaError_t Sized<float, 192>::fwd_rows(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 192>::fwd_cols(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 192>::pair_cols(const Geom&, const PipeArgs<float>&, cudaStream_t);
template int Sized<float, 192>::tm_cols(int);
template cudaError_t Sized<float, 192>::tm_max_blocks(int*);
template cudaError_t Sized<float, 192>::pair_rows_w(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 192>::rows_w_smem();
template cudaError_t Sized<float, 192>::rows_w_max_blocks(int*);
template cudaError_t Sized<float, 384>::fwd_rows(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 384>::fwd_cols(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 384>::pair_cols(const Geom&, const PipeArgs<float>&, cudaStream_t);
template int Sized<float, 384>::tm_cols(int);
template cudaError_t Sized<float, 384>::tm_max_blocks(int*);
template cudaError_t Sized<float, 384>::pair_rows_w(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 384>::rows_w_smem();
template cudaError_t Sized<float, 384>::rows_w_max_blocks(int*);
template cudaError_t Sized<float, 768>::fwd_rows(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 768>::fwd_cols(const Geom&, const PipeArgs<float>&, bool, cudaStream_t);
template cudaError_t Sized<float, 768>::pair_cols(const Geom&, const PipeArgs<float>&, cudaStream_t);
template int Sized<float, 768>::tm_cols(int);
template cudaError_t Sized<float, 768>::tm_max_blocks(int*);
template cudaError_t Sized<float, 768>::pair_rows_w(const Geom&, const PipeArgs<float>&, cudaStream_t);
template size_t Sized<float, 768>::rows_w_smem();
template cudaError_t Sized<float, 768>::rows_w_max_blocks(int*);
}
