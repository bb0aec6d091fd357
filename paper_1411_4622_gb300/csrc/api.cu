// Library-wide host utilities: error reporting and pointer classification.
#include <cstdio>
#include <string>

#include "internal.h"

namespace satpila {

namespace {
thread_local std::string g_last_error = "no error";
}

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return e == cudaErrorMemoryAllocation ? SATPILA_ERR_OOM : SATPILA_ERR_CUDA;
}

bool is_device_pointer(const void* p) {
    if (!p) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

}  // namespace satpila

extern "C" const char* satpila_last_error(void) { return satpila::g_last_error.c_str(); }

extern "C" int satpila_version(void) { return 10000; }
