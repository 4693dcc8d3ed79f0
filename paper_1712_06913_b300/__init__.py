"""B300-native MUSER imaging hot path (Mei et al., MUSER GPU imaging pipeline).

The computation lives in libmuser.so (hand-written sm_103a CUDA behind a C ABI declared
in include/muser.h); this package only marshals torch tensors to it.  Importing the
package loads the library and raises ImportError if it is missing: there is no
fallback implementation.
"""
from . import _lib
from ._lib import (ADJOINT, CALL_CENTER, CALL_CHI2, CALL_GRAD, CALL_STEER, CALL_CLEAN, CALL_DEGRID, CALL_DIRTY, CALL_GMM, CALL_GRID, CALL_IMAGE,
                   CALL_RESTORE, FORWARD, MuserError, ST_ALL_FLAGGED, ST_BEAM_FIT, ST_DROPPED, ST_GMM_DEGENERATE,
                   ST_ITER_CAP, ST_NO_DISK, ST_NONFINITE, ST_TIMEOUT)
from .api import (Config, DegridPlan, Imager, ImageResult, MixedImager, Source, Workspace, autotune, axpy, center, chi2, clean,
                  degrid, set_tuning,
                  dirty, gmm, grid, image, image_centred, CentredImager, image_side, launch_count, size_classes,
                  normalize, pixel_size, record_fields, restore, steer, uvw, workspace_size)

_lib.load()

__all__ = ["Config", "DegridPlan", "Imager", "ImageResult", "MixedImager", "Source", "image_side", "size_classes",
           "autotune", "set_tuning", "axpy", "normalize",
           "Workspace", "center", "chi2", "clean", "degrid", "dirty", "gmm", "grid", "image", "image_centred", "CentredImager",
           "launch_count", "pixel_size", "record_fields", "restore", "steer", "uvw", "workspace_size", "MuserError", "FORWARD", "ADJOINT"]
