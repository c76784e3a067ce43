// Internal interface of the learned coarse-correction network (nh_net.cu).
#pragma once
#include "nh_internal.cuh"

int nh_net_grid(nh_net n);
nh_status nh_net_forward_internal(nh_net n, const float* in, float* out);
cudaError_t kn_features(cudaStream_t st, int64_t nc, const double* rc, double inv, const float* logE, float* feat);
cudaError_t kn_from_net(cudaStream_t st, int64_t nc, const float* out, double scale, double* ec);
cudaError_t kn_inject(cudaStream_t st, int Nv, int p, int Nf, const double* ef, double inv, float* tgt);
cudaError_t kn_to_channels(cudaStream_t st, int64_t nc, const double* ec, double inv, float* t);
