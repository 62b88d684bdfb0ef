// k_spectral.cu -- Wiener-Khinchin NUFFT path (placeholder until the kernels land).
#include "spectral.cuh"

namespace ncf {

ncf_status run_spectral(const SpectralArgs &, char **, size_t *, char **, size_t *, cudaStream_t,
                        std::string *msg) {
    *msg = "spectral path not built yet";
    return NCF_EUNSUPPORTED;
}

}  // namespace ncf
