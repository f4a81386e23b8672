"""GB300-native swap-neighbourhood QAP search (2opt and tabu search walks).

The compute path is the CUDA library ``libqap.so`` (C-ABI in include/qap.h),
bound by ``_binding``; ``instances`` holds the seeded synthetic workloads.
Importing the package loads nothing; the library is built and loaded on the
first call.
"""
from ._binding import (  # noqa: F401
    EINVAL, ECUDA, ENOMEM, EOVERFLOW, ETIMEOUT, EUNSUPPORTED, FORCE_INT64, LAUNCH_PERSISTENT,
    LAUNCH_PLAIN, OK, Instance, QapError, SearchParams, Tenure, WalkOutputs, lib, make_params,
    qap_2opt, qap_cost, qap_create, qap_destroy, qap_info, qap_plan, qap_search,
    qap_search_async, qap_tabu, strerror, last_error, Batch, qap_batch_create, qap_batch_destroy,
    qap_batch_info, qap_batch_plan, qap_batch_search, qap_batch_search_async, qap_batch_autotune,
    qap_best_walks, qap_batch_set_timing, qap_batch_classes,
    qap_batch_search_noalloc, Server, qap_server_create, qap_server_destroy,
    qap_server_get_stats, qap_server_submit, qap_server_wait, TABU_PAIR, TABU_UNIT_LOC, TABU_UNIT,
    PHASE_X_AUTO, PHASE_X_DOTS,
)
