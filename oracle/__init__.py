"""FP64 CPU oracle for the splatting path -- test infrastructure only.

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import this
package.  The product path never does.
"""
