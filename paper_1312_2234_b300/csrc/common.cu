// common.cu -- error reporting of the C ABI.
#include <cstring>
#include <string>

#include "pfsi_internal.cuh"

namespace pfsi {

namespace {
thread_local std::string g_last_error;
}

int set_error(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

int check_cuda(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return PFSI_OK;
    return set_error(PFSI_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int check_launch(const char* what) { return check_cuda(cudaGetLastError(), what); }

}  // namespace pfsi

extern "C" int pfsi_last_error(char* buf, size_t len)
{
    const std::string& m = pfsi::g_last_error;
    if (buf && len > 0) {
        const size_t n = m.size() < len - 1 ? m.size() : len - 1;
        std::memcpy(buf, m.data(), n);
        buf[n] = '\0';
    }
    return (int)m.size();
}

extern "C" int pfsi_version(void) { return 100; }
