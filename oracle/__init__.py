"""FP64 CPU oracle for the sparse randomized LU path.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.
"""
from .rlu import (KEY_TAG, STATUS_OK, STATUS_WRANK, SketchParams, LUResult,
                  OracleResult, sketch_params, sem_matrix, countsketch,
                  hartley_columns, fjl, lu_partial_pivot, unit_lower,
                  pinv_householder, factor, relative_residual, check_sizes,
                  second_projection, factor_two_sketch,
                  bucket_of_word, sign_of_word, phase_of_word,
                  TRANSFORMS, hadamard_columns, srft_columns, transform_matrix,
                  column_order_greedy)
from .philox import philox4x64_10, mulhilo64, stream_blocks
