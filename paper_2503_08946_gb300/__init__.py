"""GB300-native concrete-instance SIMT race checker.

Given a kernel model with a fixed grid and parameters (threads, blocks, barrier
intervals, shared/global arrays, affine and floor-div/mod access relations), the
CUDA library expands every access instance into a packed 64-bit key, groups the
keys by cell with a onesweep radix sort, scans them for cells touched by two
threads in one barrier interval (or two blocks) with a write, and reports the
verdict, the racy-cell count and the smallest racing pair.

The public interface is the C ABI in ``include/rc.h``; ``binding`` mirrors it
in Python with the same names.  The CUDA library must be built
(``paper_2503_08946_gb300.build.build()``); there is no CPU fallback.
"""
from .binding import (RC_OK, RC_E_INVALID, RC_E_KEY_OVERFLOW, RC_E_OOB, RC_E_NOMEM, RC_E_TIMEOUT,
                      RC_E_CUDA, RC_E_NOT_READY, RC_E_UNSUPPORTED, RC_PATH_AUTO, RC_PATH_SORT,
                      RC_PATH_HASH, EXPORTS, NotReady, RcError, RcModel, RcServer, Result, check, load,
                      rc_batch_workspace_size, rc_check, rc_check_batch, rc_expand_keys, rc_get_limits,
                      rc_model_create, rc_model_create_status, rc_kernel_source, rc_model_destroy, rc_model_layout,
                      rc_report, rc_report_array, results_of, rc_sort_keys, rc_sort_keys_static, rc_sort_status, rc_ticket_stage_times, rc_sort_workspace_size, rc_status_str,
                      rc_tune, rc_workspace_size, workspace)

__all__ = [n for n in dir() if not n.startswith("_")]
