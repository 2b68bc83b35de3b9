"""GB300 (sm_103a) neural directed distance fields: batched DDF query, wavefront path tracer,
ray labelling and training, all in libddf.so's CUDA kernels behind the C ABI of include/ddf.h.

Import is cheap; the library is loaded on first use and a missing build raises ImportError
(there is no CPU fallback)."""

from ._abi import DDFError, load, LIB_PATH  # noqa: F401
from .ddf import DDFGroup, DDFNet, DDFMesh, camera_struct, measure_peaks  # noqa: F401
from .autograd import DDFFunction, ddf_apply  # noqa: F401
