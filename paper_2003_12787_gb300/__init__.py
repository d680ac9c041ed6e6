"""GB300 (sm_103a) linear ADER-DG Space-Time Predictor.

The compute lives in the CUDA library built from ``csrc/`` (C ABI:
include/stp.h); ``_binding`` marshals arguments into it and ``Predictor``
wraps a handle for torch tensors. ``inputs`` generates seeded synthetic
elastic problems.
"""
from __future__ import annotations

from ._binding import stp_ader_step, stp_correct, stp_face_params  # noqa: F401
from ._binding import (NODE_FAMILIES, PRECISIONS, STPError, stp_create,  # noqa: F401
                       stp_destroy, stp_device_status, stp_get_nodes, stp_get_precision,
                       stp_last_error,
                       stp_measure_fp64_peak, stp_measure_fp64_peak_kind, stp_nodes, stp_predict, stp_predict_host,
                       stp_predict_curvilinear, stp_predict_curvilinear_host,
                       stp_predict_sources, stp_predict_sources_curvilinear,
                       stp_reference_tables, stp_selftest_bounded_wait, stp_set_precision,
                       stp_status_string)
from ._binding import (stp_autotune, stp_batch_create, stp_batch_destroy,  # noqa: F401
                       stp_batch_info, stp_batch_launch, stp_batch_run_static,
                       stp_batch_run_static_sources)
from ._binding import (stp_server_add_sim, stp_server_create, stp_server_destroy,  # noqa: F401
                       stp_server_drain, stp_server_progress, stp_server_read,
                       stp_server_run_trace, stp_server_set_policy, stp_server_stats,
                       stp_server_submit)
from .predictor import Batch, Predictor, Server  # noqa: F401
