// Handle, device status word and error reporting of libsic.
#include <stdlib.h>

#include "sic_internal.cuh"

extern "C" sic_status sic_create(sic_handle** h, int device) {
    if (!h) return SIC_ERR_INVALID;
    *h = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return SIC_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return SIC_ERR_CUDA;
    sic_handle* p = (sic_handle*)calloc(1, sizeof(sic_handle));
    if (!p) return SIC_ERR_OOM;
    p->device = device;
    p->last_unit = -1;
    if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        free(p);
        return SIC_ERR_CUDA;
    }
    if (cudaMalloc((void**)&p->d_status, sizeof(DevStatus)) != cudaSuccess) {
        free(p);
        return SIC_ERR_OOM;
    }
    if (cudaMemset(p->d_status, 0, sizeof(DevStatus)) != cudaSuccess) {
        cudaFree(p->d_status);
        free(p);
        return SIC_ERR_CUDA;
    }
    *h = p;
    return SIC_OK;
}

extern "C" void sic_destroy(sic_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaFree(h->d_status);
    free(h);
}

extern "C" sic_status sic_sync(sic_handle* h, void* stream) {
    if (!h) return SIC_ERR_INVALID;
    SIC_CUDA_TRY(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    SIC_CUDA_TRY(cudaStreamSynchronize(s));
    DevStatus hs;
    SIC_CUDA_TRY(cudaMemcpy(&hs, h->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost));
    if (hs.code != 0) {
        h->last_unit = hs.unit;
        SIC_CUDA_TRY(cudaMemset(h->d_status, 0, sizeof(DevStatus)));
        return (sic_status)hs.code;
    }
    h->last_unit = -1;
    return SIC_OK;
}

extern "C" int64_t sic_last_error_unit(sic_handle* h) { return h ? h->last_unit : -1; }

extern "C" const char* sic_status_string(sic_status s) {
    switch (s) {
        case SIC_OK: return "ok";
        case SIC_ERR_INVALID: return "invalid argument";
        case SIC_ERR_NOT_PD: return "matrix not positive definite";
        case SIC_ERR_CUDA: return "CUDA error";
        case SIC_ERR_OOM: return "out of memory";
        case SIC_ERR_TIMEOUT: return "device wait timed out";
        case SIC_ERR_UNSUPPORTED: return "unsupported size";
    }
    return "unknown status";
}

extern "C" double sic_exhaustion_floor(const sic_kernel* kp) { return kp ? sic_floor_of(kp) : 0.0; }
