// Launch entry points of the device code, used by the host library.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "kg_internal.h"
#include "kgrape.h"

namespace kg {

constexpr int kThreads = 512;  // threads per CTA of the evaluation kernel

// kVariantGenericStream: the generic streaming loop whatever the tile size (full re-orthogonalisation)
enum { kVariantStreaming = 0, kVariantResident = 1, kVariantResidentFull = 2, kVariantGenericStream = 3 };

// Cooperative launch of the single-problem evaluation kernel (prec = kg_precision).
cudaError_t launch_eval_kernel(int prec, int variant, const EvalParams& p, int ctas, cudaStream_t stream);

// Largest co-resident grid of the evaluation kernel for a tile of 2^t_bits amplitudes.
cudaError_t eval_kernel_max_ctas(int prec, int variant, int t_bits, int* out);

// Threads per CTA of that kernel (kThreads, plus a control warp for the resident 4096-tile loop).
int eval_kernel_threads(int prec, int variant, int t_bits);

// Largest tile (log2 amplitudes) of a precision, and tiles a CTA can hold resident (0: none).
int max_tile_bits(int prec);
int resident_tiles_per_cta(int prec);

// Batched evaluation kernel (complex64): cooperative launch (CUDA-graph capturable).
cudaError_t launch_batch_kernel(const BatchParams& bp, int ctas, cudaStream_t stream);
cudaError_t batch_kernel_max_ctas(int* out);

// Record msg as the calling thread's last error (kg_last_error) and return st.
kg_status host_fail(kg_status st, const std::string& msg);

// Time limit of one pulse of a subspace launch (ns), derived from kg_set_wait_limit_ns.
long long sector_time_limit_ns();

}  // namespace kg
