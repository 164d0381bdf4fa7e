"""FP64 CPU oracle (test infrastructure only: tests, smoke check and the
bench's CPU baseline).  See ``sph_oracle`` for what it computes."""
