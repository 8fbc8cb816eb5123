// C-ABI glue: thread-local error messages, status names, descriptor defaults.
#include <string>

#include "gbx_internal.cuh"

namespace gbx {

static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }
void clear_error() { t_last_error.clear(); }

}  // namespace gbx

extern "C" const char* gbx_last_error(void) { return gbx::t_last_error.c_str(); }

extern "C" const char* gbx_status_string(gbx_status s) {
    switch (s) {
        case GBX_OK: return "GBX_OK";
        case GBX_ERR_INVALID_VALUE: return "GBX_ERR_INVALID_VALUE";
        case GBX_ERR_INVALID_INDEX: return "GBX_ERR_INVALID_INDEX";
        case GBX_ERR_DIMENSION_MISMATCH: return "GBX_ERR_DIMENSION_MISMATCH";
        case GBX_ERR_OUT_OF_MEMORY: return "GBX_ERR_OUT_OF_MEMORY";
        case GBX_ERR_NOT_SUPPORTED: return "GBX_ERR_NOT_SUPPORTED";
        case GBX_ERR_TIMEOUT: return "GBX_ERR_TIMEOUT";
        case GBX_ERR_CUDA: return "GBX_ERR_CUDA";
        case GBX_ERR_OVERFLOW: return "GBX_ERR_OVERFLOW";
        case GBX_ERR_BUSY: return "GBX_ERR_BUSY";
        case GBX_ERR_NULL_POINTER: return "GBX_ERR_NULL_POINTER";
    }
    return "GBX_ERR_UNKNOWN";
}

extern "C" int32_t gbx_version(void) { return 100; }

extern "C" void gbx_desc_init(gbx_desc* d) {
    if (!d) return;
    *d = gbx_desc{};
    d->transpose = 1;
    d->mask_complement = 0;
    d->early_exit = 1;
    d->accum = 0;
    d->direction = GBX_DIR_AUTO;
    d->heuristic = GBX_HEUR_RATIO;
    d->alpha = 0.01f;  // Section 6.3: alpha = beta = 0.01
    d->beta = 0.01f;
    d->masking = 1;
    d->operand_reuse = 1;
    d->trace = 0;
}
