"""GB300 (sm_103a) library for the contour-quadrature filter of nonlinear FEAST.

The compute path is libfeast_nl.so (CUDA, C ABI in include/feast_nl.h); this
package only builds it and binds it.
"""
from ._binding import (FeastNL, FeastError, Server, Slices, request_footprint, load_library,  # noqa: F401
                       set_contour_group,
                       strerror, last_error,
                       EXPORTS, LIB_PATH, feast_nl_term, feast_nl_info, launch_count,
                       PHASES)
from ._binding import (FEAST_NL_OK, FEAST_NL_EINVAL, FEAST_NL_ESINGULAR_NODE,  # noqa: F401
                       FEAST_NL_ENOT_CONVERGED, FEAST_NL_ETOO_MANY, FEAST_NL_ENOMEM,
                       FEAST_NL_EDEVICE, FEAST_NL_EUNSUPPORTED)
